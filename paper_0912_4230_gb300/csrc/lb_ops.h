// Host-side table of the kernels compiled for one population storage format.
// Each storage format is instantiated in its own translation unit so the
// build compiles them in parallel; the C-ABI layer picks a table at create.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbgb {

// A stored lattice for the conversion and totals kernels: element (q, n) at
// p[stride (q N + n) + off] in units of the stored type (stride 2 for the
// (f, h) pairs of 16-bit storage with solute: off 0 f, off 1 h); ref holds
// the FP16/BF16 references, a float per cell, or with ref_pair the half off
// of a __half2 per cell (NULL for FP32/FP64).
struct PopView {
  const void *p;
  int stride, off;
  const void *ref;
  int ref_pair;
};

// Record the message of a failed call that has no context; lb_last_error(NULL)
// returns it on the same thread.
void set_noctx_error(const char *msg);

// The totals kernel runs at most this many blocks (grid-stride over the
// cells), so the fixed-order finish sums few partials.
constexpr unsigned TOTALS_BLOCKS = 1024;
inline unsigned totals_blocks(unsigned nblk) { return nblk < TOTALS_BLOCKS ? nblk : TOTALS_BLOCKS; }

struct StorageOps {
  int storage;       // LB_STORE_*
  size_t elt_bytes;  // bytes per stored population
  bool fp64;         // collision type is double (StepArgs<double>)
  // step / init / rhohat take a StepArgs<Real>* matching fp64
  // feat: FEAT_OPEN (pressure / velocity faces) | FEAT_SPEC (further solute
  // species advanced by the same launch), each its own instantiation
  cudaError_t (*step)(int kmode, bool solute, int feat, const void *args, dim3 grid,
                      dim3 block, cudaStream_t s);
  // initial populations of further solute species 1 .. species-1 (u0 3N,
  // C0 species x N, device)
  cudaError_t (*species_init)(const void *args, const float *u0, const float *C0, unsigned nblk,
                              cudaStream_t s);
  cudaError_t (*init)(int kmode, bool solute, const void *args, const void *init_args,
                      unsigned nblk, cudaStream_t s);
  cudaError_t (*rhohat)(const void *args, void *rhohat, unsigned nblk, cudaStream_t s);
  // absolute FP64 populations of a lattice (0 f, 1 h) from / into storage;
  // from_f64 also sets the references (FP16/BF16). totals: FP64 sums of the
  // fluid mass and (h.p not NULL) the solute over totals_blocks(nblk) blocks,
  // one partial pair per block
  cudaError_t (*to_f64)(PopView src, double *dst, unsigned N, int lattice, cudaStream_t s);
  cudaError_t (*from_f64)(const double *src, PopView dst, unsigned N, int lattice,
                          cudaStream_t s);
  cudaError_t (*totals)(PopView f, PopView h, const uint32_t *link, unsigned N, double *partials,
                        unsigned nblk, cudaStream_t s);
  // one free-surface step, FsArgs<Real>*: five passes over the active tiles
  // (grid blocks each; the last one also lists the next step's tiles);
  // fs_seed stamps and lists the first step's tiles after initialisation (one
  // block per tile; tile_blocks is unused). NULL when the storage format has
  // no free-surface build
  cudaError_t (*fs_step)(const void *fs_args, unsigned grid, unsigned tile_blocks, cudaStream_t s);
  cudaError_t (*fs_seed)(const void *fs_args, unsigned tiles, unsigned tile_blocks, cudaStream_t s);
  // row-pipelined step kernel (NULL when not built for this storage):
  // tma_config fills the dynamic shared memory, threads per block and
  // resident blocks per SM for a row of nx cells (returns false if it does
  // not fit); tma_step launches it
  bool (*tma_config)(int kmode, bool solute, unsigned nx, size_t *smem, unsigned *threads,
                     int *blocks_per_sm);
  cudaError_t (*tma_step)(int kmode, bool solute, const void *args, unsigned grid,
                          unsigned threads, size_t smem, cudaStream_t s);
  // row-staged persistent step kernel (NULL when not built for this storage):
  // pipe_config fills the dynamic shared memory and resident blocks per SM
  // for rows of bx threads (false if it does not fit); pipe_step launches it
  // over items = gxr * ny * nz rows
  bool (*pipe_config)(int kmode, bool solute, unsigned bx, size_t *smem, int *blocks_per_sm);
  cudaError_t (*pipe_step)(int kmode, bool solute, const void *args, unsigned grid, unsigned bx,
                           size_t smem, unsigned gxr, unsigned items, cudaStream_t s);
  // one batched step: tab is a host BatchTable<Real> (passed by value in the
  // launch), work the device work list (batch_item descriptors)
  cudaError_t (*batch_step)(int kmode, bool solute, const void *tab, const uint64_t *work,
                            unsigned d_begin, unsigned vb_begin, unsigned vb_end, unsigned grid,
                            cudaStream_t s);
};

const StorageOps &ops_f32();
const StorageOps &ops_f64();
const StorageOps &ops_f16();
const StorageOps &ops_bf16();

// Setup kernels (lb_setup.cu), Real = float or double.
struct SetupArgs {
  int nx, ny, nz;
  unsigned N;
  unsigned f_wall, s_wall, s_open;  // face masks: f_wall = every non-periodic fluid face,
                                    // s_open = solute inlet | outlet faces
  const float *eps_in;   // N
  const float *K6_in;    // 6 x N packed per cell, or NULL
  const uint8_t *solid;  // N
  double D;              // solute diffusivity (0 without solute)
  void *eps;             // N Real
  void *kinv;            // 3N or 6N Real (SoA), NULL without K
  void *geps;            // 3N Real or NULL
  uint32_t *link;        // N
  unsigned *flags;       // bit 0 bad porosity, 1 K not SPD, 2 K has off-diagonals, 3 some solid
  int kmode;             // 1 diagonal, 2 full SPD (second pass)
};
cudaError_t setup_scan(const SetupArgs &a, bool fp64, cudaStream_t s);
cudaError_t setup_fields(const SetupArgs &a, bool fp64, cudaStream_t s);
cudaError_t finish_sum(const double *partials, unsigned nblk, int k, double *out, cudaStream_t s);
cudaError_t neighbors(const void *args, bool fp64, int lattice, int32_t *src, unsigned nblk,
                      cudaStream_t s);
cudaError_t fs_init(unsigned N, const uint32_t *link, const uint8_t *type_in, const float *rho0,
                    const float *lambda0, uint8_t *type0, uint8_t *type1, void *mass, void *lam,
                    bool fp64, cudaStream_t s);
cudaError_t fs_totals(unsigned N, const uint32_t *link, const void *mass, double *partials,
                      bool fp64, cudaStream_t s);
cudaError_t to_double(unsigned N, const void *src, double *dst, bool fp64, cudaStream_t s);
cudaError_t rhohat_init(unsigned N, const uint32_t *link, const float *rho0, const void *mass,
                        double wall_rho, void *rhohat, bool fp64, cudaStream_t s);

}  // namespace lbgb
