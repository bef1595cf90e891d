// Batched step: many lattices (contexts) advanced by one persistent launch per
// step.
//
// The work list is the concatenation of every lattice's blocks of the
// per-cell step kernel (same block shapes, same warp-to-flux-slot mapping),
// one 64-bit descriptor per block,
// so each lattice computes exactly what its own launch would. The grid is a
// fixed number of resident blocks that walk the list with stride gridDim.x.
// The lattices' arguments travel in the launch's parameter space
// (__grid_constant__), so the per-cell update reads them as constant-bank
// operands, as in the per-cell kernel, rather than from memory.
#pragma once

#include "lb_kernels.cuh"

namespace lbgb {

template <class Real>
struct BatchEntry {
  StepArgs<Real> a;      // arguments of the lattice's step
  unsigned gx, gy, bx;   // its per-cell launch shape: blocks along x and y, threads along x
};

// One virtual block of the work list: lattice (bits 0-15), block index along
// x (16-31), along y (32-47) and z (48-63) of the lattice's per-cell launch.
__host__ __device__ inline uint64_t batch_item(unsigned d, unsigned bxi, unsigned byi, unsigned bz) {
  return uint64_t(d) | (uint64_t(bxi) << 16) | (uint64_t(byi) << 32) | (uint64_t(bz) << 48);
}

// lattices per launch: the table stays within the 32 KB parameter space
constexpr int BATCH_MAX = 64;
template <class Real>
struct BatchTable {
  BatchEntry<Real> e[BATCH_MAX];
};
static_assert(sizeof(BatchTable<float>) <= 32000 && sizeof(BatchTable<double>) <= 32000,
              "batch table exceeds the kernel parameter space");

// Virtual blocks [vb_begin, vb_end) of the work list; item d - d_begin is
// the table entry of the block's lattice.
template <class S, int KMODE, bool SOLUTE>
__global__ void __launch_bounds__(STEP_BLOCK, 6)
    batched_step_kernel(const __grid_constant__ BatchTable<typename S::Real> tab,
                        const uint64_t *__restrict__ work, unsigned d_begin, unsigned vb_begin,
                        unsigned vb_end) {
  using Real = typename S::Real;
  for (unsigned vb = vb_begin + blockIdx.x; vb < vb_end; vb += gridDim.x) {
    const uint64_t w = __ldg(work + vb);
    const BatchEntry<Real> &e = tab.e[unsigned(w & 0xffffu) - d_begin];
    const StepArgs<Real> &a = e.a;
    const unsigned bxi = unsigned(w >> 16) & 0xffffu, byi = unsigned(w >> 32) & 0xffffu,
                   bz = unsigned(w >> 48);
    const unsigned by = STEP_BLOCK / e.bx;
    const unsigned tx = threadIdx.x & (e.bx - 1), ty = threadIdx.x / e.bx;
    const unsigned x = bxi * e.bx + tx, y = byi * by + ty, z = bz;
    const unsigned nx = a.nx, ny = a.ny;
    const unsigned warp_gid =
        ((bz * e.gy + byi) * e.gx + bxi) * (STEP_BLOCK / 32) + (threadIdx.x >> 5);
    bool live = x < nx && y < ny;
    const unsigned n = x + nx * (y + ny * z);
    uint32_t link = 0;
    if (live && a.link) {
      link = __ldg(a.link + n);
      live = !(link >> 31);
    }
    Real fin_acc = Real(0), fout_acc = Real(0), drho = Real(0), sC = Real(0);
    bool open_face = false;
    if (live)
      update_cell<S, KMODE, SOLUTE>(a, x, y, z, n, link, fin_acc, fout_acc, drho, sC, open_face);
    warp_reductions(a, warp_gid, open_face, fin_acc, fout_acc, drho, sC);
  }
}

}  // namespace lbgb
