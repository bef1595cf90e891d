// Batched step: many lattices (contexts) advanced by one persistent launch.
//
// The work list is the concatenation of every lattice's blocks of the
// per-cell step kernel (same block shapes, same warp-to-flux-slot mapping),
// so each lattice computes exactly what its own launch would. The grid is a
// fixed number of resident blocks that walk the list with stride gridDim.x.
// A one-thread-per-lattice advance kernel then swaps the population buffers
// and moves the step counter on the device, so a sequence of steps has
// constant launch arguments and can be captured once in a CUDA graph.
#pragma once

#include "lb_kernels.cuh"

namespace lbgb {

template <class Real>
struct BatchEntry {
  StepArgs<Real> a;      // arguments of the lattice's next step
  unsigned gx, gy, bx;   // its per-cell launch shape: blocks along x and y, threads along x
  unsigned blk_begin;    // first virtual block of this lattice in the work list
  float *fields;         // where the last step of the call writes the fields
  long long t_final;     // step index of the call's last step
  int check_every;
  int pad;
};
static_assert(sizeof(BatchEntry<float>) % 4 == 0 && sizeof(BatchEntry<double>) % 4 == 0,
              "batch entries are copied as 32-bit words");

template <class S, int KMODE, bool SOLUTE>
__global__ void __launch_bounds__(STEP_BLOCK, 6)
    batched_step_kernel(const BatchEntry<typename S::Real> *__restrict__ tab,
                        const uint16_t *__restrict__ owner, unsigned nd, unsigned total) {
  using Real = typename S::Real;
  // the lattice's arguments are copied to shared memory once per work item,
  // so the per-cell update reads them at shared-memory latency
  __shared__ BatchEntry<Real> se;
  constexpr unsigned words = sizeof(BatchEntry<Real>) / 4;
  for (unsigned vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const unsigned d = __ldg(owner + vb);
    __syncthreads();  // the previous item's readers are done with se
    for (unsigned w = threadIdx.x; w < words; w += blockDim.x)
      reinterpret_cast<unsigned *>(&se)[w] = __ldg(reinterpret_cast<const unsigned *>(tab + d) + w);
    __syncthreads();
    const BatchEntry<Real> &e = se;
    const StepArgs<Real> &a = e.a;
    const unsigned lb = vb - e.blk_begin;
    const unsigned bxi = lb % e.gx, byi = (lb / e.gx) % e.gy, bz = lb / (e.gx * e.gy);
    const unsigned by = STEP_BLOCK / e.bx;
    const unsigned tx = threadIdx.x % e.bx, ty = threadIdx.x / e.bx;
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

// After a batched step: swap buffers, advance t, arm the next step's flags.
template <class Real>
__global__ void batch_advance_kernel(BatchEntry<Real> *tab, unsigned nd) {
  const unsigned d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nd) return;
  StepArgs<Real> &a = tab[d].a;
  const void *fi = a.f_in;
  a.f_in = a.f_out;
  a.f_out = const_cast<void *>(fi);
  const void *hi = a.h_in;
  a.h_in = a.h_out;
  a.h_out = const_cast<void *>(hi);
  const float *rfi = a.rf_in;
  a.rf_in = a.rf_out;
  a.rf_out = const_cast<float *>(rfi);
  const float *rhi = a.rh_in;
  a.rh_in = a.rh_out;
  a.rh_out = const_cast<float *>(rhi);
  a.t += 1;
  const int ce = tab[d].check_every;
  a.reduce = (ce > 0 && a.t % ce == 0) ? 1 : 0;
  a.fields = (a.t == tab[d].t_final) ? tab[d].fields : nullptr;
}

}  // namespace lbgb
