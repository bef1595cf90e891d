// C ABI of the library (declared in include/lb.h): context management,
// validation, device memory, and the per-step launch sequence.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "lb_batch.cuh"
#include "lb_kernels.cuh"
#include "lb_ops.h"
#include "lb_tma.cuh"

using namespace lbgb;

namespace {

// process-wide allocation hooks (lb_set_allocator), read by lb_create as
// one triple under the lock, so a context never pairs one caller's alloc
// with another's user pointer
struct AllocHooks {
  void *(*alloc)(size_t, void *) = nullptr;
  void (*release)(void *, void *) = nullptr;
  void *user = nullptr;
};
AllocHooks g_hooks;
std::mutex g_hooks_mu;
thread_local std::string g_create_error;
thread_local cudaStream_t g_create_stream = nullptr;  // stream of lb_create's own work

}  // namespace

// Message of a failed call that has no context (lb_create, lb_bytes_required,
// lb_totals_noalloc), reported by lb_last_error(NULL) on the same thread.
void lbgb::set_noctx_error(const char *msg) { g_create_error = msg; }

struct lb_ctx {
  lb_domain dom{};
  lb_params prm{};
  const StorageOps *ops = nullptr;
  cudaStream_t stream = nullptr;
  unsigned N = 0, nblk = 0;
  dim3 sgrid, sblock;  // launch shape of the per-cell step kernel
  unsigned nwarps = 0;   // flux slots (one per warp of the step launch)
  bool use_tma = false;  // row-pipelined step kernel in use
  bool tma_ok = false;   // ... and available for this lattice
  unsigned tma_grid = 0, tma_threads = 0;
  size_t tma_smem = 0;
  // row-staged persistent kernel: in use when pipe.bx != 0
  struct PipeShape {
    unsigned bx = 0, grid = 0, gxr = 0, items = 0;
    size_t smem = 0;
  } pipe;
  int kmode = KM_NONE;
  bool solute = false, fs = false, has_solid = false, flux = false;
  // 16-bit storage with solute: f buffers hold (f, h) pairs of species 0, rf
  // the __half2 reference pairs, h and rh species 1 .. only
  bool paired = false;
  unsigned f_wall = 0, f_press = 0, f_vel = 0, s_wall = 0, s_inlet = 0, s_outlet = 0;
  bool open_faces = false;  // pressure or velocity faces: per-cell kernel only
  int S = 0;                // solute species (0 without the solute lattice)
  void *spec = nullptr;     // S > 1: per-species 1/tau_D, C_in, D_s/D_0 (24 Real)
  void *face = nullptr;  // per-face values of pressure / velocity faces (30 Real)
  // CUDA graphs: two steps (both buffer parities) captured once on a private
  // stream and replayed while the launch configuration holds (lb_step), and
  // the same for a batch led by this context, keyed by its members' serial
  // numbers and parities and the work list (lb_step_batch)
  bool graphs = true;
  uint64_t serial = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t g_step = nullptr;
  cudaGraphExec_t g_batch = nullptr;
  std::vector<uint64_t> g_batch_key;
  long long t = 0;
  long long n_live = 0;
  int cur = 0;
  void *f[2] = {nullptr, nullptr};
  void *h[2] = {nullptr, nullptr};
  float *rf[2] = {nullptr, nullptr};  // FP16/BF16 storage: per-cell references
  float *rh[2] = {nullptr, nullptr};
  void *eps = nullptr, *kinv = nullptr, *geps = nullptr, *rhohat = nullptr;
  uint32_t *link = nullptr;
  float *fields = nullptr;
  double *partials = nullptr;    // per-block sums of lb_reduce
  double *flux_slots = nullptr;  // per-warp cumulative inlet / outlet flux
  DevState *state = nullptr;
  // free surface
  uint8_t *type[2] = {nullptr, nullptr};
  void *mass[2] = {nullptr, nullptr};
  void *lam = nullptr, *rho_post = nullptr, *share = nullptr, *mom = nullptr;
  uint8_t *flag_a = nullptr, *flag_b = nullptr;
  unsigned *any = nullptr;
  // free surface: active-tile lists (step parity), their lengths, tile stamps
  uint32_t *tiles[2] = {nullptr, nullptr};
  unsigned *n_tiles = nullptr;
  unsigned *stamp = nullptr;
  unsigned *stamp_ctr = nullptr;  // steps taken since lb_init (device)
  unsigned ntx = 0, nty = 0, ntz = 0, fs_grid = 0;
  // table of lb_step_batch calls led by this context
  void *batch_tab = nullptr;
  size_t batch_tab_bytes = 0;
  // reusable staging for lb_init and the FP64 population exchange
  void *stage = nullptr;
  size_t stage_bytes = 0;
  std::vector<void *> allocs;
  void *(*alloc_fn)(size_t, void *) = nullptr;
  void (*release_fn)(void *, void *) = nullptr;
  void *alloc_user = nullptr;
  std::string err;
};

namespace {

int fail(lb_ctx *c, int code, const std::string &msg) {
  if (c)
    c->err = msg;
  else
    g_create_error = msg;
  return code;
}

#define CK(ctx, call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail((ctx), LB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void *dev_alloc(lb_ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (c->alloc_fn) {
    p = c->alloc_fn(bytes, c->alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->allocs.push_back(p);
  return p;
}

void dev_free(lb_ctx *c, void *p) {
  if (!p) return;
  for (size_t i = 0; i < c->allocs.size(); ++i)
    if (c->allocs[i] == p) {
      c->allocs.erase(c->allocs.begin() + i);
      break;
    }
  if (c->release_fn) {
    // A caller's allocator may hand the block out again at once (the packed
    // arena does), while launches already enqueued on the context's stream
    // (a batch work list, a graph replay) may still read it; cudaFree waits
    // by itself, a release callback does not.
    cudaStreamSynchronize(c->stream);
    c->release_fn(p, c->alloc_user);
  } else {
    cudaFree(p);
  }
}

void drop_graphs(lb_ctx *c) {
  if (c->g_step) cudaGraphExecDestroy(c->g_step);
  if (c->g_batch) cudaGraphExecDestroy(c->g_batch);
  c->g_step = c->g_batch = nullptr;
  c->g_batch_key.clear();
}

void free_all(lb_ctx *c) {
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  for (void *p : c->allocs) {
    if (c->release_fn)
      c->release_fn(p, c->alloc_user);
    else
      cudaFree(p);
  }
  c->allocs.clear();
}

void *stage(lb_ctx *c, size_t bytes) {
  if (c->stage_bytes >= bytes) return c->stage;
  dev_free(c, c->stage);
  c->stage = dev_alloc(c, bytes);
  c->stage_bytes = c->stage ? bytes : 0;
  return c->stage;
}

unsigned face_mask(const int32_t (&k)[3][2], int kind) {
  unsigned m = 0;
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s)
      if (k[a][s] == kind) m |= 1u << (2 * a + s);
  return m;
}

const StorageOps *ops_of(int storage) {
  switch (storage) {
    case LB_STORE_FP32: return &ops_f32();
    case LB_STORE_FP64: return &ops_f64();
    case LB_STORE_FP16DEV: return &ops_f16();
    case LB_STORE_BF16DEV: return &ops_bf16();
    default: return nullptr;
  }
}

// Launch shape of the per-cell step kernel: rows of BX threads (a multiple
// of 32, up to the lattice width), BY rows per block.
void cell_shape(const lb_domain &dom, dim3 *grid, dim3 *block) {
  unsigned bx = 32;
  while (bx < unsigned(STEP_BLOCK) && bx < unsigned(dom.nx)) bx *= 2;
  *block = dim3(bx, STEP_BLOCK / bx, 1);
  *grid = dim3((dom.nx + bx - 1) / bx, (dom.ny + block->y - 1) / block->y, dom.nz);
}

// Flux slots: one pair per warp of the widest launch any step kernel may
// take. The per-cell kernel's launches over every row width bound the
// others: the row-pipelined grid has at most ny nz blocks of nx/32 warps, and
// the row-staged grid with rows of bx threads at most ceil(nx/bx) ny nz
// blocks of bx/32 warps, which the per-cell launch with rows of bx covers.
unsigned slot_warps(const lb_domain &dom) {
  unsigned w = 0;
  for (unsigned bx = 32; bx <= unsigned(STEP_BLOCK); bx *= 2) {
    const unsigned by = STEP_BLOCK / bx;
    w = std::max(w, ((dom.nx + bx - 1) / bx) * ((dom.ny + by - 1) / by) * dom.nz *
                        (STEP_BLOCK / 32));
  }
  return w;
}

// Device memory of one lattice, block by block, as lb_create and lb_init
// allocate it; one function, so that lb_bytes_required reports what the
// allocation does. k_rows: rows of K^-1 kept (0, 3 diagonal, 6 full tensor).
struct Layout {
  size_t f, h, rf, rh;   // per population buffer (two of each; 0 = not allocated)
  size_t spec;           // several species: per-species constants
  size_t eps, link, fields, partials, state, geps, rhohat, face;
  size_t fs_type, fs_mass, fs_lam, fs_rho, fs_share, fs_mom, fs_flag, fs_any, fs_tiles, fs_ntiles,
      fs_stamp, fs_stamp_ctr;
  size_t kinv, flux_slots;
  size_t create_stage;   // inputs of lb_create, released before it returns
  size_t init_stage;     // inputs of lb_init, kept for later staging
  size_t batch_share;    // this lattice's part of a batch work list (lb_step_batch)
};

Layout layout_of(const lb_domain &dom, const lb_params &prm, const StorageOps &ops, int k_rows,
                 bool f_scale) {
  Layout L{};
  const size_t N = size_t(dom.nx) * dom.ny * dom.nz;
  const size_t rb = ops.fp64 ? 8 : 4;
  const size_t pb = size_t(Q) * N * ops.elt_bytes;
  const bool shift = (prm.storage == LB_STORE_FP16DEV || prm.storage == LB_STORE_BF16DEV);
  const bool solute = prm.solute != 0;
  const size_t S = solute ? size_t(std::max(1, int(prm.species))) : 1;
  const bool paired = shift && solute;
  // species held in the h buffers (the paired layout keeps species 0 with f)
  const size_t Sh = solute ? S - (paired ? 1 : 0) : 0;
  L.f = paired ? 2 * pb : pb;
  L.h = Sh * pb;
  // a float per cell, or the __half2 reference pair of the paired layout
  L.rf = shift ? N * sizeof(float) : 0;
  L.rh = (shift && Sh) ? S * N * sizeof(float) : 0;
  if (solute && S > 1) {
    L.spec = 24 * rb;
  }
  L.eps = N * rb;
  L.link = N * 4;
  L.fields = (5 + S) * N * sizeof(float);  // rho, u (3), C, nu, then C of species 1 .. S-1
  const size_t nblk = (N + BLOCK - 1) / BLOCK;
  L.partials = nblk * 4 * sizeof(double);
  L.state = sizeof(DevState);
  L.geps = solute ? 3 * N * rb : 0;
  L.rhohat = (prm.A != 0.0 || prm.free_surface) ? N * rb : 0;
  L.face = 30 * rb;
  if (prm.free_surface) {
    const size_t ntiles = size_t((unsigned(dom.nx) + FS_TX - 1) / FS_TX) *
                          ((unsigned(dom.ny) + FS_TY - 1) / FS_TY) *
                          ((unsigned(dom.nz) + FS_TZ - 1) / FS_TZ);
    L.fs_type = N;
    L.fs_mass = N * rb;
    L.fs_lam = N * rb;
    L.fs_rho = N * rb;
    L.fs_share = N * rb;
    L.fs_mom = 4 * N * rb;
    L.fs_flag = N;
    L.fs_any = sizeof(unsigned);
    L.fs_tiles = ntiles * sizeof(uint32_t);
    L.fs_ntiles = 2 * sizeof(unsigned);
    L.fs_stamp = ntiles * sizeof(unsigned);
    L.fs_stamp_ctr = sizeof(unsigned);
  }
  L.kinv = size_t(k_rows) * N * rb;
  L.flux_slots = size_t(slot_warps(dom)) * 2 * S * sizeof(double);
  L.create_stage = N * 4 + (k_rows ? 6 * N * 4 : 0) + N + 64 + 256;
  L.init_stage = N * 4 * (4 + S) + (f_scale ? size_t(Q) * N * 4 : 0) + N * 4 + N + 256;
  dim3 g, b;
  cell_shape(dom, &g, &b);
  L.batch_share = size_t(g.x) * g.y * g.z * sizeof(uint64_t);
  return L;
}

// Bytes of a block as a caller's allocator with 256-byte granules (the
// packed arena) accounts for it; dev_alloc takes at least 16 bytes.
size_t granule(size_t b) { return b == 0 ? 0 : (std::max<size_t>(b, 16) + 255) / 256 * 256; }

template <class Real>
void fill_args(const lb_ctx *c, StepArgs<Real> &a) {
  std::memset(&a, 0, sizeof a);
  a.nx = c->dom.nx;
  a.ny = c->dom.ny;
  a.nz = c->dom.nz;
  a.N = c->N;
  a.f_wall = c->f_wall;
  a.f_press = c->f_press;
  a.f_vel = c->f_vel;
  a.face = static_cast<const Real *>(c->face);
  a.spec = static_cast<const Real *>(c->spec);
  a.species = c->S;
  a.slot_stride = c->nwarps * 2;
  a.s_wall = c->s_wall;
  a.s_inlet = c->s_inlet;
  a.s_outlet = c->s_outlet;
  a.f_in = c->f[c->cur];
  a.f_out = c->f[1 - c->cur];
  a.h_in = c->h[c->cur];
  a.h_out = c->h[1 - c->cur];
  a.rf_in = c->rf[c->cur];
  a.rf_out = c->rf[1 - c->cur];
  a.rh_in = c->rh[c->cur];
  a.rh_out = c->rh[1 - c->cur];
  a.paired = c->paired ? 1 : 0;
  a.eps = static_cast<const Real *>(c->eps);
  a.kinv = static_cast<const Real *>(c->kinv);
  a.geps = static_cast<const Real *>(c->geps);
  a.link = c->has_solid ? c->link : nullptr;
  a.rhohat = static_cast<const Real *>(c->rhohat);
  for (int i = 0; i < 3; ++i) a.G[i] = Real(c->prm.G[i]);
  a.tau = Real(c->prm.tau);
  a.tau0 = Real(c->prm.tau0);
  a.tau1 = Real(c->prm.tau1);
  a.nu_g = Real(c->prm.nu_g);
  a.a_h = Real(c->prm.a);
  a.alpha = Real(c->prm.alpha);
  a.beta = Real(c->prm.beta);
  a.visc_law = c->prm.visc_law;
  a.A = Real(c->prm.A);
  a.wall_rho = Real(c->prm.wall_rho);
  a.forch = Real(c->prm.forchheimer);
  if (c->solute) {
    a.inv_tau_D = Real(1.0 / c->prm.tau_D);
    a.D = Real((c->prm.tau_D - 0.5) / 3.0);
    a.C_in = Real(c->prm.C_in);
  }
  a.t = c->t;
  a.flux = c->flux ? 1 : 0;
  a.flux_slots = c->flux_slots;
  a.state = c->state;
}

// Run fn(args) with StepArgs of the context's collision type.
template <class Fn>
int with_args(lb_ctx *c, Fn &&fn) {
  if (c->ops->fp64) {
    StepArgs<double> a;
    fill_args(c, a);
    return fn(static_cast<void *>(&a), a);
  }
  StepArgs<float> a;
  fill_args(c, a);
  return fn(static_cast<void *>(&a), a);
}

int check_status(lb_ctx *c) {
  DevState st;
  CK(c, cudaMemcpyAsync(&st, c->state, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (st.status & 2u) return fail(c, LB_ETIMEOUT, "a bounded wait of the step kernel gave up");
  if (st.status & 1u) return fail(c, LB_ENONFINITE, "a step reduction met a NaN or an infinity");
  return LB_OK;
}

// Launch shape of the row-staged kernel for rows of bx threads: the grid is
// the resident blocks of all SMs, at most one block per row.
bool pipe_shape(const lb_ctx *c, unsigned bx, lb_ctx::PipeShape *ps) {
  if (!c->ops->pipe_config || c->open_faces || c->S > 1) return false;
  size_t smem = 0;
  int bps = 0, sms = 0, dev = 0;
  const bool ok = c->ops->pipe_config(c->kmode, c->solute, bx, &smem, &bps) &&
                  cudaGetDevice(&dev) == cudaSuccess &&
                  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
  cudaGetLastError();
  if (!ok) return false;
  ps->bx = bx;
  ps->gxr = (unsigned(c->dom.nx) + bx - 1) / bx;
  ps->items = ps->gxr * unsigned(c->dom.ny) * unsigned(c->dom.nz);
  ps->grid = std::min(ps->items, unsigned(bps) * unsigned(sms));
  ps->smem = smem;
  return ps->grid * (bx / 32) <= c->nwarps;  // within the flux slots (always, by slot_warps)
}

// Free-surface arguments of the step that brings the state to step index t
// (t = 0: the arguments that seed the first step's tiles).
template <class Real>
FsArgs<Real> fs_args(lb_ctx *c, const StepArgs<Real> &a, long long t) {
  FsArgs<Real> fa;
  fa.a = a;
  fa.a.fields = c->fields;  // rho and V' of every live cell feed the re-typing
  fa.a.link = c->link;
  fa.type_old = c->type[c->cur];
  fa.type_new = c->type[1 - c->cur];
  fa.m_old = static_cast<Real *>(c->mass[c->cur]);
  fa.m_new = static_cast<Real *>(c->mass[1 - c->cur]);
  fa.lam = static_cast<Real *>(c->lam);
  fa.rhohat_w = static_cast<Real *>(c->rhohat);
  fa.flag_a = c->flag_a;
  fa.flag_b = c->flag_b;
  fa.rho_post = static_cast<Real *>(c->rho_post);
  fa.share = static_cast<Real *>(c->share);
  fa.mom = static_cast<Real *>(c->mom);
  fa.any = c->any;
  fa.tiles = c->tiles[t & 1];
  fa.n_tiles = c->n_tiles + (t & 1);
  fa.next_tiles = c->tiles[(t + 1) & 1];
  fa.next_n_tiles = c->n_tiles + ((t + 1) & 1);
  fa.stamp = c->stamp;
  fa.stamp_ctr = c->stamp_ctr;
  fa.ntx = c->ntx;
  fa.nty = c->nty;
  fa.ntz = c->ntz;
  return fa;
}

// The current populations of the fluid lattice and of solute species sp as
// stored (the paired layout keeps f and species 0 in one buffer).
PopView f_view(const lb_ctx *c) {
  return PopView{c->f[c->cur], c->paired ? 2 : 1, 0, c->rf[c->cur], c->paired ? 1 : 0};
}
PopView h_view(const lb_ctx *c, int sp) {
  if (c->paired && sp == 0) return PopView{c->f[c->cur], 2, 1, c->rf[c->cur], 1};
  const size_t hoff = size_t(sp - (c->paired ? 1 : 0)) * Q * c->N * c->ops->elt_bytes;
  const float *rh = c->rh[c->cur] ? c->rh[c->cur] + size_t(sp) * c->N : nullptr;
  return PopView{static_cast<const char *>(c->h[c->cur]) + hoff, 1, 0, rh, 0};
}

unsigned fs_tile_count(const lb_ctx *c) { return c->ntx * c->nty * c->ntz; }

// features of the per-cell step kernel this lattice needs
int step_feat(const lb_ctx *c);

// One step of a lattice (the one that brings it to t + 1 from buffer parity
// cur) enqueued on stream s; with last the step exports the fields. Launches
// only, so it can be captured into a graph.
int enqueue_step(lb_ctx *c, cudaStream_t s, bool last) {
  return with_args(c, [&](void *args, auto &a) {
    using Real = std::remove_reference_t<decltype(a.G[0])>;
    a.t = c->t + 1;
    a.reduce = (c->prm.check_every > 0 && a.t % c->prm.check_every == 0) ? 1 : 0;
    a.fields = last ? c->fields : nullptr;
    if (c->fs) {
      a.fields = c->fields;
      const FsArgs<Real> fa = fs_args(c, a, a.t);
      CK(c, c->ops->fs_step(&fa, c->fs_grid, (fs_tile_count(c) + BLOCK - 1) / BLOCK, s));
      return int(LB_OK);
    }
    if (c->prm.A != 0.0) CK(c, c->ops->rhohat(args, c->rhohat, c->nblk, s));
    if (c->use_tma)
      CK(c, c->ops->tma_step(c->kmode, c->solute, args, c->tma_grid, c->tma_threads, c->tma_smem, s));
    else if (c->pipe.bx)
      CK(c, c->ops->pipe_step(c->kmode, c->solute, args, c->pipe.grid, c->pipe.bx, c->pipe.smem,
                              c->pipe.gxr, c->pipe.items, s));
    else {
      CK(c, c->ops->step(c->kmode, c->solute, step_feat(c), args, c->sgrid, c->sblock, s));
    }
    return int(LB_OK);
  });
}

// A lattice's steps can be replayed from a graph when every step of a pair
// launches the same work with the same arguments: no time-dependent viscosity
// (t is an argument) and checks on every step or none. (The free surface's
// tile lists and stamps live on the device, its passes' grids are fixed.)
bool graph_safe(const lb_ctx *c) {
  return c->graphs && c->prm.visc_law != 2 && c->prm.check_every <= 1;
}

// Capture two steps, issued by step(stream) with the lattices' t and parity
// advanced in between (enqueue restores nothing: the caller's step function
// reads c->t / c->cur), on the leader's private stream, and instantiate.
template <class StepFn, class AdvanceFn>
int capture_two(lb_ctx *lead, cudaGraphExec_t *out, StepFn &&step, AdvanceFn &&advance) {
  if (!lead->cap_stream &&
      cudaStreamCreateWithFlags(&lead->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return LB_ECUDA;
  }
  if (cudaStreamBeginCapture(lead->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return LB_ECUDA;
  }
  int rc = step(lead->cap_stream);
  advance(+1);
  if (rc == LB_OK) rc = step(lead->cap_stream);
  advance(-1);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(lead->cap_stream, &g);
  if (rc == LB_OK && e == cudaSuccess && g &&
      cudaGraphInstantiate(out, g, 0) == cudaSuccess) {
    cudaGraphDestroy(g);
    return LB_OK;
  }
  if (g) cudaGraphDestroy(g);
  *out = nullptr;
  cudaGetLastError();
  return LB_ECUDA;
}

template <class StepFn>
int capture_pair(lb_ctx *c, cudaGraphExec_t *out, StepFn &&step) {
  return capture_two(c, out, step, [&](int d) {
    c->t += d;
    c->cur = 1 - c->cur;
  });
}

// features of the per-cell step kernel this lattice needs
int step_feat(const lb_ctx *c) { return (c->open_faces ? FEAT_OPEN : 0) | (c->S > 1 ? FEAT_SPEC : 0); }

// One warp waits, with the step kernels' bounded wait, on a shared-memory
// barrier that nothing completes; on giving up it sets the timeout bit of the
// context's status word, as the row-pipelined kernel does.
__global__ void wait_timeout_kernel(DevState *state, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncwarp();
  mbar_fence_init();
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar, 0, limit_ns));
  if (!ok && threadIdx.x == 0) atomicOr(&state->status, 2u);
}

// fluid faces: PERIODIC, WALL, PRESSURE, VELOCITY; solute faces: PERIODIC,
// WALL, INLET, OUTLET
bool valid_faces(const int32_t (&k)[3][2], bool fluid) {
  for (int a = 0; a < 3; ++a) {
    for (int s = 0; s < 2; ++s) {
      const int v = k[a][s];
      if (fluid ? !(v == LB_BC_PERIODIC || v == LB_BC_WALL || v == LB_BC_PRESSURE ||
                    v == LB_BC_VELOCITY)
                : (v < 0 || v > 3))
        return false;
    }
    if ((k[a][0] == LB_BC_PERIODIC) != (k[a][1] == LB_BC_PERIODIC)) return false;
  }
  return true;
}

}  // namespace

extern "C" {

int lb_set_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *user) {
  if ((alloc == nullptr) != (release == nullptr)) return LB_EINVAL;
  std::lock_guard<std::mutex> lock(g_hooks_mu);
  g_hooks.alloc = alloc;
  g_hooks.release = release;
  g_hooks.user = user;
  return LB_OK;
}

int lb_bytes_required(const lb_domain *dom, const lb_params *prm, int32_t k_rows,
                      int32_t f_scale, size_t *bytes) {
  if (!dom || !prm || !bytes) return fail(nullptr, LB_EINVAL, "domain, params and bytes are required");
  *bytes = 0;
  if (dom->nx < 1 || dom->ny < 1 || dom->nz < 1)
    return fail(nullptr, LB_EINVAL, "lattice size out of range");
  if (k_rows != 0 && k_rows != 3 && k_rows != 6)
    return fail(nullptr, LB_EINVAL, "k_rows must be 0, 3 or 6");
  const StorageOps *ops = ops_of(prm->storage);
  if (!ops) return fail(nullptr, LB_EINVAL, "storage");
  if (prm->species < 0 || prm->species > LB_MAX_SPECIES)
    return fail(nullptr, LB_EINVAL, "species outside [0, LB_MAX_SPECIES]");
  const Layout L = layout_of(*dom, *prm, *ops, k_rows, f_scale != 0);
  const size_t twice[] = {L.f, L.h, L.rf, L.rh, L.fs_type, L.fs_mass, L.fs_flag, L.fs_tiles};
  const size_t once[] = {L.spec, L.eps, L.link, L.fields, L.partials, L.state, L.geps,
                         L.rhohat, L.face, L.fs_lam, L.fs_rho, L.fs_share, L.fs_mom, L.fs_any,
                         L.fs_ntiles, L.fs_stamp, L.fs_stamp_ctr, L.kinv, L.flux_slots,
                         L.batch_share};
  size_t total = 0;
  for (size_t b : twice) total += 2 * granule(b);
  for (size_t b : once) total += granule(b);
  // the creation inputs are released before lb_init takes its staging block
  total += std::max(granule(L.create_stage), granule(L.init_stage));
  *bytes = total;
  return LB_OK;
}

int lb_create(const lb_domain *dom, const float *porosity, const float *K6, const uint8_t *solid,
              const lb_params *prm, lb_ctx **out) {
  if (!out) return fail(nullptr, LB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!dom || !porosity || !solid || !prm)
    return fail(nullptr, LB_EINVAL, "domain, porosity, solid and params are required");
  const long long N64 = (long long)dom->nx * dom->ny * dom->nz;
  if (dom->nx < 1 || dom->ny < 1 || dom->nz < 1 || dom->nz > 65535)
    return fail(nullptr, LB_EINVAL, "lattice size out of range (nz <= 65535)");
  if (19 * N64 > 0x7fffffffLL)
    return fail(nullptr, LB_EUNSUPPORTED, "lattice too large: 19 N must stay below 2^31");
  if (!valid_faces(dom->bc, true) || !valid_faces(dom->sbc, false))
    return fail(nullptr, LB_EINVAL, "invalid face kinds");
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s)
      if (dom->bc[a][s] == LB_BC_WALL && dom->sbc[a][s] != LB_BC_WALL)
        return fail(nullptr, LB_EINVAL, "solute faces must be WALL where the fluid has a wall");
  if (!(prm->forchheimer >= 0.0)) return fail(nullptr, LB_EINVAL, "forchheimer < 0");
  if (prm->visc_law < 0 || prm->visc_law > 2) return fail(nullptr, LB_EINVAL, "visc_law");
  if (prm->visc_law == 0 && !(prm->tau > 0.5)) return fail(nullptr, LB_EINVAL, "tau <= 1/2");
  if (prm->visc_law == 1 && !(prm->tau0 > 0.5 && prm->tau1 > 0.5))
    return fail(nullptr, LB_EINVAL, "tau0, tau1 <= 1/2");
  if (prm->visc_law == 2 && !(prm->nu_g > 0.0)) return fail(nullptr, LB_EINVAL, "nu_g <= 0");
  if (prm->visc_law != 0 && !prm->solute)
    return fail(nullptr, LB_EINVAL, "a concentration-dependent viscosity needs the solute lattice");
  if (prm->solute && !(prm->tau_D > 0.5)) return fail(nullptr, LB_EINVAL, "tau_D <= 1/2");
  if (prm->species < 0 || prm->species > LB_MAX_SPECIES)
    return fail(nullptr, LB_EINVAL, "species outside [0, LB_MAX_SPECIES]");
  if (prm->species > 1 && !prm->solute)
    return fail(nullptr, LB_EINVAL, "several species need the solute lattice");
  for (int sp = 1; sp < prm->species; ++sp)
    if (!(prm->species_tau_D[sp] > 0.5)) return fail(nullptr, LB_EINVAL, "species tau_D <= 1/2");
  if (prm->free_surface && (prm->solute || K6))
    return fail(nullptr, LB_EUNSUPPORTED, "free surface with solute or permeability");
  if ((face_mask(dom->bc, LB_BC_PRESSURE) | face_mask(dom->bc, LB_BC_VELOCITY)) &&
      (prm->free_surface || prm->A != 0.0))
    return fail(nullptr, LB_EUNSUPPORTED,
                "pressure / velocity faces with a free surface or surface tension");
  if (prm->check_every < 0) return fail(nullptr, LB_EINVAL, "check_every < 0");
  if (prm->kernel < 0 || prm->kernel > 3) return fail(nullptr, LB_EINVAL, "kernel");
  const StorageOps *ops = ops_of(prm->storage);
  if (!ops) return fail(nullptr, LB_EINVAL, "storage");
  if (prm->free_surface && !ops->fs_step)
    return fail(nullptr, LB_EUNSUPPORTED, "free surface is not built for this storage");

  lb_ctx *c = new (std::nothrow) lb_ctx;
  if (!c) return fail(nullptr, LB_ENOMEM, "host allocation");
  static std::atomic<uint64_t> next_serial{1};
  c->serial = next_serial++;
  c->dom = *dom;
  c->prm = *prm;
  c->ops = ops;
  c->stream = g_create_stream;
  {
    std::lock_guard<std::mutex> lock(g_hooks_mu);
    c->alloc_fn = g_hooks.alloc;
    c->release_fn = g_hooks.release;
    c->alloc_user = g_hooks.user;
  }
  c->N = unsigned(N64);
  c->nblk = (c->N + BLOCK - 1) / BLOCK;
  cell_shape(*dom, &c->sgrid, &c->sblock);
  c->nwarps = slot_warps(*dom);  // flux slots for every launch shape the autotuner may pick
  c->solute = prm->solute != 0;
  c->fs = prm->free_surface != 0;
  c->f_wall = face_mask(dom->bc, LB_BC_WALL);
  c->f_press = face_mask(dom->bc, LB_BC_PRESSURE);
  c->f_vel = face_mask(dom->bc, LB_BC_VELOCITY);
  c->open_faces = (c->f_press | c->f_vel) != 0;
  c->s_wall = face_mask(dom->sbc, LB_BC_WALL);
  c->s_inlet = c->solute ? face_mask(dom->sbc, LB_BC_INLET) : 0;
  c->s_outlet = c->solute ? face_mask(dom->sbc, LB_BC_OUTLET) : 0;
  c->flux = (c->s_inlet | c->s_outlet) != 0;
  auto bail = [&](int code) {
    std::string m = c->err;
    free_all(c);
    delete c;
    g_create_error = m;
    return code;
  };
  const size_t N = c->N;
  const size_t rb = ops->fp64 ? 8 : 4;
  // device memory, block by block as layout_of lists it
  const Layout L = layout_of(*dom, *prm, *ops, K6 ? 6 : 0, false);
  const bool shift = (prm->storage == LB_STORE_FP16DEV || prm->storage == LB_STORE_BF16DEV);
  c->S = c->solute ? std::max(1, int(prm->species)) : 0;
  c->paired = shift && c->solute;
  for (int b = 0; b < 2; ++b) {
    if (!(c->f[b] = dev_alloc(c, L.f))) return bail(fail(c, LB_ENOMEM, "populations f"));
    if (L.h && !(c->h[b] = dev_alloc(c, L.h))) return bail(fail(c, LB_ENOMEM, "populations h"));
    if (L.rf && !(c->rf[b] = static_cast<float *>(dev_alloc(c, L.rf))))
      return bail(fail(c, LB_ENOMEM, "references"));
    if (L.rh && !(c->rh[b] = static_cast<float *>(dev_alloc(c, L.rh))))
      return bail(fail(c, LB_ENOMEM, "references"));
  }
  if (c->S > 1) {
    double sv[24] = {};
    const double D0 = (prm->tau_D - 0.5) / 3.0;
    for (int sp = 0; sp < c->S; ++sp) {
      const double tD = sp ? prm->species_tau_D[sp] : prm->tau_D;
      sv[sp] = 1.0 / tD;
      sv[8 + sp] = sp ? prm->species_C_in[sp] : prm->C_in;
      sv[16 + sp] = ((tD - 0.5) / 3.0) / D0;
    }
    if (!(c->spec = dev_alloc(c, L.spec)))
      return bail(fail(c, LB_ENOMEM, "species"));
    float sf[24];
    for (int i = 0; i < 24; ++i) sf[i] = float(sv[i]);
    cudaError_t e = cudaMemcpyAsync(c->spec, rb == 8 ? static_cast<const void *>(sv) : sf,
                                    24 * rb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // host arrays leave scope
    if (e != cudaSuccess)
      return bail(fail(c, LB_ECUDA, std::string("species values: ") + cudaGetErrorString(e)));
  }
  c->eps = dev_alloc(c, L.eps);
  c->link = static_cast<uint32_t *>(dev_alloc(c, L.link));
  c->fields = static_cast<float *>(dev_alloc(c, L.fields));
  c->partials = static_cast<double *>(dev_alloc(c, L.partials));
  c->state = static_cast<DevState *>(dev_alloc(c, L.state));
  if (!c->eps || !c->link || !c->fields || !c->partials || !c->state)
    return bail(fail(c, LB_ENOMEM, "static fields"));
  if (L.geps && !(c->geps = dev_alloc(c, L.geps))) return bail(fail(c, LB_ENOMEM, "geps"));
  if (L.rhohat && !(c->rhohat = dev_alloc(c, L.rhohat)))
    return bail(fail(c, LB_ENOMEM, "rhohat"));
  {
    // per-face values: 3 x pressure (the face density over eps), velocity,
    // and the part of 3 x pressure below the collision type's rounding (the
    // face density rho_b = 3 eps P sits near 1, and the flow it drives follows
    // rho_b - 1, which the rounded 3P alone would carry to only ~1e-7)
    double fv[30] = {};
    for (int f = 0; f < 6; ++f) {
      fv[f] = 3.0 * prm->face_P[f / 2][f % 2];
      for (int i = 0; i < 3; ++i) fv[6 + 3 * f + i] = prm->face_u[f / 2][f % 2][i];
      if (rb == 4) fv[24 + f] = fv[f] - double(float(fv[f]));
    }
    if (!(c->face = dev_alloc(c, L.face))) return bail(fail(c, LB_ENOMEM, "face values"));
    float ff[30];
    for (int i = 0; i < 30; ++i) ff[i] = float(fv[i]);
    cudaError_t e = cudaMemcpyAsync(c->face, rb == 8 ? static_cast<const void *>(fv) : ff,
                                    30 * rb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // host arrays leave scope
    if (e != cudaSuccess)
      return bail(fail(c, LB_ECUDA, std::string("face values: ") + cudaGetErrorString(e)));
  }
  if (c->fs) {
    for (int b = 0; b < 2; ++b) {
      c->type[b] = static_cast<uint8_t *>(dev_alloc(c, L.fs_type));
      c->mass[b] = dev_alloc(c, L.fs_mass);
      if (!c->type[b] || !c->mass[b]) return bail(fail(c, LB_ENOMEM, "free surface"));
    }
    c->lam = dev_alloc(c, L.fs_lam);
    c->rho_post = dev_alloc(c, L.fs_rho);
    c->share = dev_alloc(c, L.fs_share);
    c->mom = dev_alloc(c, L.fs_mom);
    c->flag_a = static_cast<uint8_t *>(dev_alloc(c, L.fs_flag));
    c->flag_b = static_cast<uint8_t *>(dev_alloc(c, L.fs_flag));
    c->any = static_cast<unsigned *>(dev_alloc(c, L.fs_any));
    c->ntx = (unsigned(dom->nx) + FS_TX - 1) / FS_TX;
    c->nty = (unsigned(dom->ny) + FS_TY - 1) / FS_TY;
    c->ntz = (unsigned(dom->nz) + FS_TZ - 1) / FS_TZ;
    const size_t ntiles = size_t(c->ntx) * c->nty * c->ntz;
    c->tiles[0] = static_cast<uint32_t *>(dev_alloc(c, L.fs_tiles));
    c->tiles[1] = static_cast<uint32_t *>(dev_alloc(c, L.fs_tiles));
    c->n_tiles = static_cast<unsigned *>(dev_alloc(c, L.fs_ntiles));
    c->stamp = static_cast<unsigned *>(dev_alloc(c, L.fs_stamp));
    c->stamp_ctr = static_cast<unsigned *>(dev_alloc(c, L.fs_stamp_ctr));
    if (!c->lam || !c->rho_post || !c->share || !c->mom || !c->flag_a || !c->flag_b || !c->any || !c->tiles[0] ||
        !c->tiles[1] || !c->n_tiles || !c->stamp || !c->stamp_ctr)
      return bail(fail(c, LB_ENOMEM, "free surface"));
    // persistent grid of the tile passes: enough resident blocks to cover
    // the list of a typical step in one round
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return bail(fail(c, LB_ECUDA, "device attributes"));
    c->fs_grid = unsigned(std::min<size_t>(ntiles, size_t(FS_BLOCKS_PER_SM) * unsigned(sms)));
  }
  // inputs -> device (caller pointers may be host or device)
  const size_t in_bytes = N * 4 + (K6 ? 6 * N * 4 : 0) + N + 64;
  char *in = static_cast<char *>(dev_alloc(c, L.create_stage));  // in_bytes + 256
  if (!in) return bail(fail(c, LB_ENOMEM, "staging"));
  float *eps_in = reinterpret_cast<float *>(in);
  float *K_in = K6 ? eps_in + N : nullptr;
  uint8_t *sol_in = reinterpret_cast<uint8_t *>(in + N * 4 + (K6 ? 6 * N * 4 : 0));
  unsigned *flags = reinterpret_cast<unsigned *>(in + ((in_bytes + 15) & ~size_t(15)));
  int rc = LB_OK;
  auto ck = [&](cudaError_t e, const char *what) {
    if (e != cudaSuccess && rc == LB_OK) rc = fail(c, LB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  ck(cudaMemcpyAsync(eps_in, porosity, N * 4, cudaMemcpyDefault, c->stream), "copy porosity");
  if (K6) ck(cudaMemcpyAsync(K_in, K6, 6 * N * 4, cudaMemcpyDefault, c->stream), "copy K");
  ck(cudaMemcpyAsync(sol_in, solid, N, cudaMemcpyDefault, c->stream), "copy solid");
  ck(cudaMemsetAsync(flags, 0, sizeof(unsigned), c->stream), "memset");
  ck(cudaMemsetAsync(c->state, 0, sizeof(DevState), c->stream), "memset");
  if (rc != LB_OK) return bail(rc);
  SetupArgs sa{};
  sa.nx = dom->nx;
  sa.ny = dom->ny;
  sa.nz = dom->nz;
  sa.N = c->N;
  sa.f_wall = c->f_wall | c->f_press | c->f_vel;  // links only to cells inside or wrapped
  sa.s_wall = c->s_wall;
  sa.s_open = face_mask(dom->sbc, LB_BC_INLET) | face_mask(dom->sbc, LB_BC_OUTLET);
  sa.eps_in = eps_in;
  sa.K6_in = K_in;
  sa.solid = sol_in;
  sa.D = c->solute ? (prm->tau_D - 0.5) / 3.0 : 0.0;
  sa.flags = flags;
  ck(setup_scan(sa, ops->fp64, c->stream), "setup scan");
  unsigned hflags = 0;
  ck(cudaMemcpyAsync(&hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, c->stream), "flags");
  ck(cudaStreamSynchronize(c->stream), "sync");
  if (rc != LB_OK) return bail(rc);
  if (hflags & 1u) return bail(fail(c, LB_EINVAL, "porosity outside (0, 1] in a non-solid cell"));
  if (hflags & 2u) return bail(fail(c, LB_EINVAL, "permeability tensor not positive definite"));
  c->has_solid = (hflags & 8u) != 0;
  c->kmode = !K6 ? KM_NONE : ((hflags & 4u) ? KM_SPD : KM_DIAG);
  if (c->kmode == KM_SPD && prm->forchheimer != 0.0)
    return bail(fail(c, LB_EUNSUPPORTED, "Forchheimer drag needs a diagonal permeability tensor"));
  if (c->kmode == KM_DIAG && prm->forchheimer != 0.0) c->kmode = KM_FORCH;
  if (K6 && !(c->kinv = dev_alloc(c, layout_of(*dom, *prm, *ops, c->kmode == KM_SPD ? 6 : 3,
                                                 false).kinv)))
    return bail(fail(c, LB_ENOMEM, "K inverse"));
  // row-pipelined kernel: eligible shapes only; grid = resident blocks of all SMs
  // (automatic selection keeps the per-cell kernel: on GB300 at 128^3 it is
  // 2x faster than this row-pipelined form, which stays available on request)
  if (prm->kernel != 1 && !c->fs && !c->open_faces && c->S <= 1 && ops->tma_config) {
    int bps = 0, sms = 0, dev = 0;
    if (ops->tma_config(c->kmode, c->solute, unsigned(dom->nx), &c->tma_smem, &c->tma_threads,
                        &bps) &&
        cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
      const unsigned rows = unsigned(dom->ny) * unsigned(dom->nz);
      c->tma_grid = std::min(rows, unsigned(bps) * unsigned(sms));
      // the flux slots cover its warps (slot_warps bounds every launch shape)
      c->tma_ok = c->tma_grid * unsigned(dom->nx / 32) <= c->nwarps;
      c->use_tma = c->tma_ok && prm->kernel == 2;
    }
    cudaGetLastError();
  }
  if (prm->kernel == 2 && !c->use_tma)
    return bail(fail(c, LB_EUNSUPPORTED, "row-pipelined kernel: this lattice shape or storage"));
  if (prm->kernel == 3) {
    const unsigned bx = c->sblock.x;
    if (c->fs || !ops->pipe_config || !pipe_shape(c, bx, &c->pipe))
      return bail(fail(c, LB_EUNSUPPORTED, "row-staged kernel: this lattice or storage"));
  }
  c->flux_slots = static_cast<double *>(dev_alloc(c, L.flux_slots));
  if (!c->flux_slots) return bail(fail(c, LB_ENOMEM, "flux slots"));
  sa.eps = c->eps;
  sa.kinv = c->kinv;
  sa.geps = c->geps;
  sa.link = c->link;
  sa.kmode = c->kmode;
  ck(setup_fields(sa, ops->fp64, c->stream), "setup fields");
  ck(cudaStreamSynchronize(c->stream), "sync");
  if (rc != LB_OK) return bail(rc);
  dev_free(c, in);
  std::vector<uint8_t> hs(N);
  // count of live cells, for the mass of the in-step check
  if (cudaMemcpyAsync(hs.data(), solid, N, cudaMemcpyDefault, c->stream) == cudaSuccess &&
      cudaStreamSynchronize(c->stream) == cudaSuccess) {
    long long live = 0;
    for (size_t i = 0; i < N; ++i) live += hs[i] == 0;
    c->n_live = live;
  }
  *out = c;
  return LB_OK;
}

int lb_set_stream(lb_ctx *c, void *stream) {
  if (!c) {
    g_create_stream = static_cast<cudaStream_t>(stream);
    return LB_OK;
  }
  c->stream = static_cast<cudaStream_t>(stream);
  return LB_OK;
}

int lb_init(lb_ctx *c, const float *rho0, const float *u0, const float *C0,
            const uint8_t *cell_type, const float *lambda0, const float *f_scale) {
  if (!c) return LB_EINVAL;
  if (!rho0 || !u0) return fail(c, LB_EINVAL, "rho0 and u0 are required");
  if (c->solute && !C0) return fail(c, LB_EINVAL, "C0 is required with the solute lattice");
  if (c->fs && !cell_type) return fail(c, LB_EINVAL, "cell_type is required with a free surface");
  const size_t N = c->N;
  const size_t S = size_t(std::max(c->S, 1));  // C0: N values per species
  const size_t bytes = layout_of(c->dom, c->prm, *c->ops, 0, f_scale != nullptr).init_stage;
  char *st = static_cast<char *>(stage(c, bytes));
  if (!st) return fail(c, LB_ENOMEM, "staging");
  float *d_rho = reinterpret_cast<float *>(st);
  float *d_u = d_rho + N;
  float *d_C = d_u + 3 * N;
  float *d_lam = d_C + S * N;
  float *d_fs = d_lam + N;
  uint8_t *d_type = reinterpret_cast<uint8_t *>(d_fs + (f_scale ? size_t(Q) * N : 0));
  // Inputs the GPU can address (device, managed, pinned or registered host
  // memory) are read in place by the initialisation kernels; the others are
  // copied to the staging block first.
  auto in_place = [](const void *p) -> const void * {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
    if (at.type == cudaMemoryTypeHost) return at.devicePointer;
    return nullptr;
  };
  {
    const void *v = in_place(rho0);
    if (v) d_rho = const_cast<float *>(static_cast<const float *>(v));
    else CK(c, cudaMemcpyAsync(d_rho, rho0, N * 4, cudaMemcpyDefault, c->stream));
    v = in_place(u0);
    if (v) d_u = const_cast<float *>(static_cast<const float *>(v));
    else CK(c, cudaMemcpyAsync(d_u, u0, 3 * N * 4, cudaMemcpyDefault, c->stream));
    if (C0) {
      v = in_place(C0);
      if (v) d_C = const_cast<float *>(static_cast<const float *>(v));
      else CK(c, cudaMemcpyAsync(d_C, C0, S * N * 4, cudaMemcpyDefault, c->stream));
    }
    if (f_scale) {
      v = in_place(f_scale);
      if (v) d_fs = const_cast<float *>(static_cast<const float *>(v));
      else CK(c, cudaMemcpyAsync(d_fs, f_scale, size_t(Q) * N * 4, cudaMemcpyDefault, c->stream));
    }
  }
  if (c->fs) {
    CK(c, cudaMemcpyAsync(d_type, cell_type, N, cudaMemcpyDefault, c->stream));
    if (lambda0) CK(c, cudaMemcpyAsync(d_lam, lambda0, N * 4, cudaMemcpyDefault, c->stream));
  }
  c->t = 0;
  c->cur = 0;
  CK(c, cudaMemsetAsync(c->state, 0, sizeof(DevState), c->stream));
  CK(c, cudaMemsetAsync(c->flux_slots, 0,
                        size_t(c->nwarps) * 2 * size_t(std::max(c->S, 1)) * sizeof(double),
                        c->stream));
  if (c->fs) {
    CK(c, fs_init(c->N, c->link, d_type, d_rho, lambda0 ? d_lam : nullptr, c->type[0], c->type[1],
                  c->mass[0], c->lam, c->ops->fp64, c->stream));
    CK(c, rhohat_init(c->N, c->link, d_rho, c->mass[0], c->prm.wall_rho, c->rhohat, c->ops->fp64,
                      c->stream));
    // cells outside the active tiles are never written by a step: both mass
    // buffers and both flag arrays start equal (no flag), no tile is stamped
    const size_t rb = c->ops->fp64 ? 8 : 4;
    CK(c, cudaMemcpyAsync(c->mass[1], c->mass[0], N * rb, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemsetAsync(c->flag_a, 0, N, c->stream));
    CK(c, cudaMemsetAsync(c->flag_b, 0, N, c->stream));
    CK(c, cudaMemsetAsync(c->stamp, 0, size_t(fs_tile_count(c)) * sizeof(unsigned), c->stream));
    CK(c, cudaMemsetAsync(c->stamp_ctr, 0, sizeof(unsigned), c->stream));
    CK(c, cudaMemsetAsync(c->n_tiles, 0, 2 * sizeof(unsigned), c->stream));
  } else if (c->prm.A != 0.0) {
    CK(c, rhohat_init(c->N, c->link, d_rho, nullptr, c->prm.wall_rho, c->rhohat, c->ops->fp64,
                      c->stream));
  }
  return with_args(c, [&](void *args, auto &a) {
    using Real = std::remove_reference_t<decltype(a.G[0])>;
    a.link = c->link;  // solid cells are always skipped at init
    a.t = 0;
    a.fields = c->fields;
    InitArgs<Real> in{};
    in.rho0 = d_rho;
    in.u0 = d_u;
    in.C0 = C0 ? d_C : nullptr;
    in.f_scale = f_scale ? d_fs : nullptr;
    in.type = c->fs ? c->type[0] : nullptr;
    CK(c, c->ops->init(c->kmode, c->solute, args, &in, c->nblk, c->stream));
    if (c->S > 1) CK(c, c->ops->species_init(args, d_u, d_C, c->nblk, c->stream));
    if (c->fs) {  // the first step's active tiles
      const FsArgs<Real> fa = fs_args(c, a, 0);
      CK(c, c->ops->fs_seed(&fa, fs_tile_count(c), (fs_tile_count(c) + BLOCK - 1) / BLOCK,
                            c->stream));
    }
    return int(LB_OK);
  });
}

int lb_step(lb_ctx *c, int64_t n) {
  if (!c) return LB_EINVAL;
  if (n < 0) return fail(c, LB_EINVAL, "n < 0");
  int64_t i = 0;
  while (i < n) {
    // all but the last step (which exports the fields) in whole pairs from
    // the graph, starting from buffer parity 0
    const int64_t pairs = (n - i - 1) / 2;
    if (pairs > 0 && c->cur == 0 && graph_safe(c)) {
      if (!c->g_step && capture_pair(c, &c->g_step, [&](cudaStream_t s) {
            return enqueue_step(c, s, false);
          }) != LB_OK)
        c->graphs = false;  // not capturable here: plain launches from now on
      if (c->g_step) {
        for (int64_t p = 0; p < pairs; ++p) CK(c, cudaGraphLaunch(c->g_step, c->stream));
        c->t += 2 * pairs;
        i += 2 * pairs;
        continue;
      }
    }
    const int rc = enqueue_step(c, c->stream, i == n - 1);
    if (rc != LB_OK) return rc;
    c->t += 1;
    c->cur = 1 - c->cur;
    ++i;
  }
  return LB_OK;
}

int lb_debug_graphs(const lb_ctx *c) {
  if (!c) return LB_EINVAL;
  return (c->g_step ? 1 : 0) | (c->g_batch ? 2 : 0);
}

int lb_set_graphs(lb_ctx *c, int32_t enable) {
  if (!c) return LB_EINVAL;
  CK(c, cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  c->graphs = enable != 0;
  return LB_OK;
}

}  // extern "C"

namespace {

template <class Real>
int step_batch_t(lb_ctx *const *ctxs, int n, int64_t steps) {
  lb_ctx *c0 = ctxs[0];
  if (n > 65535) return fail(c0, LB_EUNSUPPORTED, "more than 65535 lattices in one batch");
  int dev = 0, sms = 0;
  CK(c0, cudaGetDevice(&dev));
  CK(c0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned wave = unsigned(6 * sms);  // resident blocks of the per-cell kernel
  // a lattice whose own launch fills the GPU steps alone (its per-cell launch);
  // the smaller ones share the persistent launches, their blocks concatenated
  std::vector<int> alone, shared;
  for (int i = 0; i < n; ++i) {
    const dim3 g = ctxs[i]->sgrid;
    (g.x * g.y * g.z >= wave || ctxs[i]->open_faces || ctxs[i]->S > 1 ? alone : shared)
        .push_back(i);
  }
  const int ns = int(shared.size());
  std::vector<unsigned> begin(size_t(ns) + 1);
  unsigned total = 0;
  for (int j = 0; j < ns; ++j) {
    const dim3 g = ctxs[shared[j]]->sgrid;
    begin[j] = total;
    total += g.x * g.y * g.z;
  }
  begin[ns] = total;
  cudaStream_t s = c0->stream;
  const uint64_t *d_work = nullptr;
  if (ns > 0) {
    std::vector<uint64_t> work(total);
    for (int j = 0; j < ns; ++j) {
      const dim3 g = ctxs[shared[j]]->sgrid;
      unsigned b = begin[j];
      for (unsigned bz = 0; bz < g.z; ++bz)
        for (unsigned by = 0; by < g.y; ++by)
          for (unsigned bx = 0; bx < g.x; ++bx) work[b++] = batch_item(unsigned(j), bx, by, bz);
    }
    const size_t wbytes = work.size() * sizeof(uint64_t);
    if (c0->batch_tab_bytes < wbytes) {
      dev_free(c0, c0->batch_tab);
      c0->batch_tab = dev_alloc(c0, wbytes);
      c0->batch_tab_bytes = c0->batch_tab ? wbytes : 0;
      if (!c0->batch_tab) return fail(c0, LB_ENOMEM, "batch work list");
    }
    d_work = static_cast<const uint64_t *>(c0->batch_tab);
    CK(c0, cudaMemcpyAsync(c0->batch_tab, work.data(), wbytes, cudaMemcpyHostToDevice, s));
  }
  // one table per launch of at most BATCH_MAX lattices, filled on the host
  // for every step (the launch copies it into its parameter space)
  std::unique_ptr<BatchTable<Real>> tab(new BatchTable<Real>());
  auto one_step = [&](cudaStream_t st, bool last) -> int {
    auto step_args = [&](lb_ctx *c, StepArgs<Real> &a) {
      fill_args(c, a);
      a.t = c->t + 1;
      a.reduce = (c->prm.check_every > 0 && a.t % c->prm.check_every == 0) ? 1 : 0;
      a.fields = last ? c->fields : nullptr;
    };
    for (int i : alone) {
      StepArgs<Real> a;
      step_args(ctxs[i], a);
      CK(c0, c0->ops->step(c0->kmode, c0->solute, step_feat(ctxs[i]), &a, ctxs[i]->sgrid,
                           ctxs[i]->sblock, st));
    }
    for (int g0 = 0; g0 < ns; g0 += BATCH_MAX) {
      const int g1 = std::min(ns, g0 + BATCH_MAX);
      std::memset(tab.get(), 0, sizeof(BatchTable<Real>));
      for (int j = g0; j < g1; ++j) {
        lb_ctx *c = ctxs[shared[j]];
        BatchEntry<Real> &e = tab->e[j - g0];
        step_args(c, e.a);
        e.gx = c->sgrid.x;
        e.gy = c->sgrid.y;
        e.bx = c->sblock.x;
      }
      const unsigned blocks = begin[g1] - begin[g0];
      CK(c0, c0->ops->batch_step(c0->kmode, c0->solute, tab.get(), d_work, unsigned(g0),
                                 begin[g0], begin[g1], std::min(blocks, wave), st));
    }
    return int(LB_OK);
  };
  auto advance = [&](int d) {
    for (int i = 0; i < n; ++i) {
      ctxs[i]->t += d;
      ctxs[i]->cur = 1 - ctxs[i]->cur;
    }
  };
  // the graph of a step pair is valid for this set of lattices in this order,
  // these parities and this work list
  bool safe = true;
  std::vector<uint64_t> key;
  key.push_back(uint64_t(reinterpret_cast<uintptr_t>(d_work)));
  for (int i = 0; i < n; ++i) {
    safe = safe && graph_safe(ctxs[i]);
    key.push_back(ctxs[i]->serial * 2 + uint64_t(ctxs[i]->cur));
  }
  int64_t k = 0;
  const int64_t pairs = steps > 0 ? (steps - 1) / 2 : 0;
  if (safe && pairs > 0) {
    if (!c0->g_batch || c0->g_batch_key != key) {
      if (c0->g_batch) cudaGraphExecDestroy(c0->g_batch);
      c0->g_batch = nullptr;
      c0->g_batch_key.clear();
      if (capture_two(c0, &c0->g_batch, [&](cudaStream_t st) { return one_step(st, false); },
                      advance) == LB_OK)
        c0->g_batch_key = key;
    }
    if (c0->g_batch) {
      for (int64_t p = 0; p < pairs; ++p) CK(c0, cudaGraphLaunch(c0->g_batch, s));
      for (int i = 0; i < n; ++i) ctxs[i]->t += 2 * pairs;
      k = 2 * pairs;
    }
  }
  for (; k < steps; ++k) {
    const int rc = one_step(s, k == steps - 1);
    if (rc != LB_OK) return rc;
    advance(+1);
  }
  return LB_OK;
}

}  // namespace

extern "C" {

int lb_step_batch(lb_ctx *const *ctxs, int32_t n, int64_t steps) {
  if (!ctxs || n < 1 || steps < 0) return LB_EINVAL;
  lb_ctx *c0 = ctxs[0];
  if (!c0) return LB_EINVAL;
  for (int i = 0; i < n; ++i) {
    lb_ctx *c = ctxs[i];
    if (!c) return fail(c0, LB_EINVAL, "NULL context in batch");
    if (c->ops != c0->ops || c->kmode != c0->kmode || c->solute != c0->solute)
      return fail(c0, LB_EUNSUPPORTED, "batch lattices must share storage, permeability mode and solute");
    if (c->fs || c->prm.A != 0.0)
      return fail(c0, LB_EUNSUPPORTED, "batch: free surface and surface tension step alone");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(c0, LB_EINVAL, "context twice in one batch");
  }
  if (steps == 0) return LB_OK;
  return c0->ops->fp64 ? step_batch_t<double>(ctxs, n, steps) : step_batch_t<float>(ctxs, n, steps);
}

int lb_debug_wait_timeout(lb_ctx *c, int64_t limit_ns) {
  if (!c) return LB_EINVAL;
  if (limit_ns < 1 || limit_ns > 2000000000LL) return fail(c, LB_EINVAL, "limit_ns outside (0, 2 s]");
  wait_timeout_kernel<<<1, 32, 0, c->stream>>>(c->state, (unsigned long long)limit_ns);
  CK(c, cudaGetLastError());
  return check_status(c);
}

int lb_autotune(lb_ctx *c, int32_t reps, int32_t *choice) {
  if (!c) return LB_EINVAL;
  if (reps < 1) reps = 1;
  if (choice) *choice = 0;
  if (c->fs || c->prm.A != 0.0) return LB_OK;  // fixed launches (free surface, surface tension)
  enum Kind { CELL, ROWS, STAGED };
  struct Cand {
    Kind kind;
    unsigned bx;
    lb_ctx::PipeShape ps;
  };
  std::vector<Cand> cands;
  for (unsigned bx = 32; bx <= unsigned(STEP_BLOCK); bx *= 2) cands.push_back({CELL, bx, {}});
  if (c->tma_ok) cands.push_back({ROWS, 0, {}});
  for (unsigned bx = 32; bx <= unsigned(STEP_BLOCK); bx *= 2) {
    Cand cd{STAGED, bx, {}};
    if (pipe_shape(c, bx, &cd.ps)) cands.push_back(cd);
  }
  cudaEvent_t e0, e1;
  CK(c, cudaEventCreate(&e0));
  CK(c, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_i = -1;
  int rc = LB_OK;
  for (size_t i = 0; i < cands.size() && rc == LB_OK; ++i) {
    const Cand &cd = cands[i];
    const dim3 blk(cd.bx, STEP_BLOCK / std::max(cd.bx, 1u), 1);
    const dim3 grd(cd.bx ? (c->dom.nx + blk.x - 1) / blk.x : 1,
                   cd.bx ? (c->dom.ny + blk.y - 1) / blk.y : 1, c->dom.nz);
    // side-effect free timing launches: input buffer -> output buffer without
    // swapping, no flux accumulation, no checks, no field export
    auto launch = [&]() -> int {
      return with_args(c, [&](void *args, auto &a) {
        a.t = c->t + 1;
        a.flux = 0;
        a.reduce = 0;
        a.fields = nullptr;
        if (cd.kind == ROWS)
          CK(c, c->ops->tma_step(c->kmode, c->solute, args, c->tma_grid, c->tma_threads,
                                 c->tma_smem, c->stream));
        else if (cd.kind == STAGED)
          CK(c, c->ops->pipe_step(c->kmode, c->solute, args, cd.ps.grid, cd.ps.bx, cd.ps.smem,
                                  cd.ps.gxr, cd.ps.items, c->stream));
        else
          CK(c, c->ops->step(c->kmode, c->solute, step_feat(c), args, grd, blk, c->stream));
        return int(LB_OK);
      });
    };
    rc = launch();  // warm-up
    if (rc != LB_OK) break;
    if (cudaEventRecord(e0, c->stream) != cudaSuccess) {
      rc = fail(c, LB_ECUDA, "autotune event");
      break;
    }
    for (int r = 0; r < reps && rc == LB_OK; ++r) rc = launch();
    if (rc != LB_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = fail(c, LB_ECUDA, "autotune timing");
      break;
    }
    if (ms < best) {
      best = ms;
      best_i = int(i);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LB_OK || best_i < 0) return rc;
  const Cand &w = cands[best_i];
  drop_graphs(c);  // the captured launches used the previous shape
  c->use_tma = w.kind == ROWS;
  c->pipe = w.kind == STAGED ? w.ps : lb_ctx::PipeShape{};
  if (w.kind == CELL) {
    c->sblock = dim3(w.bx, STEP_BLOCK / w.bx, 1);
    c->sgrid = dim3((c->dom.nx + w.bx - 1) / w.bx, (c->dom.ny + c->sblock.y - 1) / c->sblock.y,
                    c->dom.nz);
  }
  if (choice) *choice = w.kind == ROWS ? 256 : (w.kind == STAGED ? 1000 + int(w.bx) : int(w.bx));
  return LB_OK;
}

int lb_fields(lb_ctx *c, float *rho, float *u, float *C, float *nu) {
  if (!c) return LB_EINVAL;
  const size_t N = c->N;
  if (rho) CK(c, cudaMemcpyAsync(rho, c->fields, N * 4, cudaMemcpyDefault, c->stream));
  if (u) CK(c, cudaMemcpyAsync(u, c->fields + N, 3 * N * 4, cudaMemcpyDefault, c->stream));
  if (C) CK(c, cudaMemcpyAsync(C, c->fields + 4 * N, N * 4, cudaMemcpyDefault, c->stream));
  if (nu) CK(c, cudaMemcpyAsync(nu, c->fields + 5 * N, N * 4, cudaMemcpyDefault, c->stream));
  return check_status(c);
}

int lb_reduce(lb_ctx *c, double *mass, double *solute, double *flux_in, double *flux_out) {
  if (!c) return LB_EINVAL;
  double *out = static_cast<double *>(stage(c, 64));
  if (!out) return fail(c, LB_ENOMEM, "staging");
  double tot[4] = {0.0, 0.0, 0.0, 0.0};
  if (c->fs)
    CK(c, fs_totals(c->N, c->link, c->mass[c->cur], c->partials, c->ops->fp64, c->stream));
  else
    CK(c, c->ops->totals(f_view(c), c->solute ? h_view(c, 0) : PopView{},
                         c->has_solid ? c->link : nullptr, c->N, c->partials, c->nblk, c->stream));
  CK(c, finish_sum(c->partials, c->fs ? c->nblk : totals_blocks(c->nblk), 2, out, c->stream));
  CK(c, finish_sum(c->flux_slots, c->nwarps, 2, out + 2, c->stream));
  CK(c, cudaMemcpyAsync(tot, out, sizeof tot, cudaMemcpyDeviceToHost, c->stream));
  DevState st;
  CK(c, cudaMemcpyAsync(&st, c->state, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (mass) *mass = tot[0];
  if (solute) *solute = tot[1];
  if (flux_in) *flux_in = tot[2];
  if (flux_out) *flux_out = tot[3];
  if (st.status & 1u) return fail(c, LB_ENONFINITE, "a step reduction met a NaN or an infinity");
  return LB_OK;
}

int lb_species_state(lb_ctx *c, int32_t sp, float *C, double *totals, double *h) {
  if (!c) return LB_EINVAL;
  if (sp < 0 || sp >= c->S) return fail(c, LB_EINVAL, "no such solute species");
  const size_t N = c->N;
  const PopView hv = h_view(c, sp);
  if (C) {
    const float *src = c->fields + (sp == 0 ? 4 * N : (5 + size_t(sp)) * N);
    CK(c, cudaMemcpyAsync(C, src, N * sizeof(float), cudaMemcpyDefault, c->stream));
  }
  if (totals) {
    double *out = static_cast<double *>(stage(c, 64));
    if (!out) return fail(c, LB_ENOMEM, "staging");
    CK(c, c->ops->totals(f_view(c), hv, c->has_solid ? c->link : nullptr, c->N, c->partials,
                         c->nblk, c->stream));
    CK(c, finish_sum(c->partials, totals_blocks(c->nblk), 2, out, c->stream));
    CK(c, finish_sum(c->flux_slots + size_t(sp) * c->nwarps * 2, c->nwarps, 2, out + 2,
                     c->stream));
    double tot[4];
    CK(c, cudaMemcpyAsync(tot, out, sizeof tot, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    totals[0] = tot[1];
    totals[1] = tot[2];
    totals[2] = tot[3];
  }
  if (h) {
    double *st = static_cast<double *>(stage(c, size_t(Q) * N * sizeof(double)));
    if (!st) return fail(c, LB_ENOMEM, "staging");
    CK(c, c->ops->to_f64(hv, st, c->N, 1, c->stream));
    CK(c, cudaMemcpyAsync(h, st, size_t(Q) * N * sizeof(double), cudaMemcpyDefault, c->stream));
  }
  return check_status(c);
}

int lb_set_populations(lb_ctx *c, const double *f, const double *h) {
  if (!c) return LB_EINVAL;
  const size_t N = c->N;
  double *st = static_cast<double *>(stage(c, size_t(Q) * N * sizeof(double)));
  if (!st) return fail(c, LB_ENOMEM, "staging");
  if (f) {
    CK(c, cudaMemcpyAsync(st, f, size_t(Q) * N * 8, cudaMemcpyDefault, c->stream));
    CK(c, c->ops->from_f64(st, f_view(c), c->N, 0, c->stream));
  }
  if (h && c->solute) {
    CK(c, cudaMemcpyAsync(st, h, size_t(Q) * N * 8, cudaMemcpyDefault, c->stream));
    CK(c, c->ops->from_f64(st, h_view(c, 0), c->N, 1, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

int lb_get_populations(lb_ctx *c, double *f, double *h) {
  if (!c) return LB_EINVAL;
  const size_t N = c->N;
  double *st = static_cast<double *>(stage(c, size_t(Q) * N * sizeof(double)));
  if (!st) return fail(c, LB_ENOMEM, "staging");
  if (f) {
    CK(c, c->ops->to_f64(f_view(c), st, c->N, 0, c->stream));
    CK(c, cudaMemcpyAsync(f, st, size_t(Q) * N * 8, cudaMemcpyDefault, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  if (h && c->solute) {
    CK(c, c->ops->to_f64(h_view(c, 0), st, c->N, 1, c->stream));
    CK(c, cudaMemcpyAsync(h, st, size_t(Q) * N * 8, cudaMemcpyDefault, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  return LB_OK;
}

int lb_debug_neighbors(lb_ctx *c, int32_t lattice, int32_t *src) {
  if (!c || !src || lattice < 0 || lattice > 1) return c ? fail(c, LB_EINVAL, "arguments") : LB_EINVAL;
  const size_t N = c->N;
  int32_t *st = static_cast<int32_t *>(stage(c, size_t(Q) * N * 4));
  if (!st) return fail(c, LB_ENOMEM, "staging");
  const int rc = with_args(c, [&](void *args, auto &a) {
    a.link = c->link;
    CK(c, neighbors(args, c->ops->fp64, lattice, st, c->nblk, c->stream));
    return int(LB_OK);
  });
  if (rc != LB_OK) return rc;
  CK(c, cudaMemcpyAsync(src, st, size_t(Q) * N * 4, cudaMemcpyDefault, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

int lb_free_surface_state(lb_ctx *c, uint8_t *type, double *mass) {
  if (!c) return LB_EINVAL;
  if (!c->fs) return fail(c, LB_EINVAL, "no free surface in this context");
  const size_t N = c->N;
  if (type) CK(c, cudaMemcpyAsync(type, c->type[c->cur], N, cudaMemcpyDefault, c->stream));
  if (mass) {
    double *st = static_cast<double *>(stage(c, N * sizeof(double)));
    if (!st) return fail(c, LB_ENOMEM, "staging");
    CK(c, to_double(c->N, c->mass[c->cur], st, c->ops->fp64, c->stream));
    CK(c, cudaMemcpyAsync(mass, st, N * sizeof(double), cudaMemcpyDefault, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

int lb_sync(lb_ctx *c) {
  if (!c) return LB_EINVAL;
  return check_status(c);
}

int64_t lb_time(const lb_ctx *c) { return c ? c->t : -1; }

const char *lb_last_error(const lb_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void lb_destroy(lb_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

}  // extern "C"
