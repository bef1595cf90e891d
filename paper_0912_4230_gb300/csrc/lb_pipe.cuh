// Row-staged persistent step kernel (FP32 and FP64 storage).
//
// The per-cell kernel issues all of a cell's loads, waits for them and then
// computes; while a warp computes it has no loads in flight, so at the
// register-limited occupancy the memory system idles part of the time. Here
// each block owns a row segment of BX cells at a time and walks the rows
// (x-block, y, z) with stride gridDim.x. While a thread computes its cell of
// row r, cp.async copies everything its cell of row r + gridDim.x will read
// (the 19 pulled f, the 19 pulled h, D grad(eps)/eps, eps, the K^-1 rows,
// the link word) into the thread's own column of a second shared-memory
// stage, so every warp keeps loads in flight while it computes. A thread
// reads only the column it wrote, so cp.async.wait_group alone orders the
// stages; no block barrier is needed.
//
// Not used for lattices with pressure or velocity faces. Cells next to a
// bounce-back link, a wall face or an open solute face take
// the per-cell path (update_cell) with its own global loads; the staged
// values of such cells are not used. Every staged address is the wrapped
// pull source of a cell inside the lattice, so it is in bounds for any cell.
// The arithmetic of a cell is the per-cell kernel's (fluid_moments and
// collide_tail), so both kernels give the same results.
#pragma once

#include "lb_kernels.cuh"

namespace lbgb {

template <class S, int KMODE, bool SOLUTE>
struct PipeLayout {
  using Real = typename S::Real;
  static_assert(sizeof(typename S::T) == sizeof(Real), "staged rows are copied element by element");
  static constexpr int kKinv = KMODE == KM_SPD ? 6 : (KMODE == KM_NONE ? 0 : 3);
  // rows of one stage: f [0, Q), h [Q, 2Q), D grad(eps)/eps (3), eps, K^-1
  static constexpr int kH = Q;
  static constexpr int kGeps = SOLUTE ? 2 * Q : Q;
  static constexpr int kEps = kGeps + (SOLUTE ? 3 : 0);
  static constexpr int kKin = kEps + 1;
  static constexpr int kRows = kKin + kKinv;
  // two stages of kRows x bx values and two stages of bx link words
  static size_t smem_bytes(unsigned bx) {
    return 2 * (size_t(kRows) * bx * sizeof(Real) + size_t(bx) * sizeof(uint32_t));
  }
};

template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Launch: blockDim.x = bx (32, 64 or 128), dynamic shared memory
// PipeLayout::smem_bytes(bx), any grid; items = gxr * ny * nz rows with gxr =
// ceil(nx / bx). Flux slots: one per warp of the launch.
template <class S, int KMODE, bool SOLUTE>
__global__ void __launch_bounds__(STEP_BLOCK, 4)
    pipe_step_kernel(const StepArgs<typename S::Real> a, unsigned gxr, unsigned items) {
  using Real = typename S::Real;
  using T = typename S::T;
  using L = PipeLayout<S, KMODE, SOLUTE>;
  extern __shared__ __align__(16) unsigned char pipe_smem[];
  const unsigned bx = blockDim.x, tid = threadIdx.x;
  Real *const sv = reinterpret_cast<Real *>(pipe_smem);                    // [2][kRows][bx]
  uint32_t *const sl = reinterpret_cast<uint32_t *>(sv + 2 * L::kRows * bx);  // [2][bx]
  const unsigned nx = a.nx, ny = a.ny, nz = a.nz, N = a.N;
  const unsigned warp_gid = blockIdx.x * (bx >> 5) + (tid >> 5);

  auto stage = [&](unsigned it, unsigned s) {
    if (it >= items) return;
    const unsigned r = it / gxr;
    const unsigned x = (it - r * gxr) * bx + tid, y = r % ny, z = r / ny;
    if (x >= nx) return;
    const unsigned n = x + nx * (y + ny * z);
    const CellGeo g = cell_geo_xyz(x, y, z, nx, ny, nz);
    Real *const dst = sv + size_t(s) * L::kRows * bx + tid;
    const T *const fb = static_cast<const T *>(a.f_in) + n;
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      cp_async<sizeof(Real)>(dst + q * bx, fb + (int(q * N) + src_delta<q>(g)));
    });
    if (SOLUTE) {
      const T *const hb = static_cast<const T *>(a.h_in) + n;
      Unroll<0, Q>::run([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        cp_async<sizeof(Real)>(dst + (L::kH + q) * bx, hb + (int(q * N) + src_delta<q>(g)));
      });
      for (int k = 0; k < 3; ++k)
        cp_async<sizeof(Real)>(dst + (L::kGeps + k) * bx, a.geps + size_t(k) * N + n);
    }
    cp_async<sizeof(Real)>(dst + L::kEps * bx, a.eps + n);
    for (int k = 0; k < L::kKinv; ++k)
      cp_async<sizeof(Real)>(dst + (L::kKin + k) * bx, a.kinv + size_t(k) * N + n);
    if (a.link) cp_async<4>(sl + s * bx + tid, a.link + n);
  };

  unsigned s = 0;
  stage(blockIdx.x, 0);
  cp_async_commit();
  for (unsigned it = blockIdx.x; it < items; it += gridDim.x) {
    stage(it + gridDim.x, s ^ 1u);
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of row `it` have landed
    const unsigned r = it / gxr;
    const unsigned x = (it - r * gxr) * bx + tid, y = r % ny, z = r / ny;
    const unsigned n = x + nx * (y + ny * z);
    bool live = x < nx;
    uint32_t link = 0;
    if (live && a.link) {
      link = sl[s * bx + tid];
      live = !(link >> 31);
    }
    Real fin_acc = Real(0), fout_acc = Real(0), drho = Real(0), sC = Real(0);
    bool open_face = false;
    if (live) {
      const CellGeo g = cell_geo_xyz(x, y, z, nx, ny, nz);
      const bool simple = link == 0 && !(g.onface & a.f_wall) &&
                          (!SOLUTE || !(g.onface & (a.s_wall | a.s_inlet | a.s_outlet)));
      if (simple) {
        const Real *const src = sv + size_t(s) * L::kRows * bx + tid;
        Real d[Q];
        Unroll<0, Q>::run([&](auto qc) { d[decltype(qc)::value] = src[decltype(qc)::value * bx]; });
        const Real eps = src[L::kEps * bx];
        Real gx = Real(0), gy = Real(0), gz = Real(0);
        if (SOLUTE) {
          gx = src[L::kGeps * bx];
          gy = src[(L::kGeps + 1) * bx];
          gz = src[(L::kGeps + 2) * bx];
          Unroll<0, Q>::run([&](auto qc) { sC += src[(L::kH + decltype(qc)::value) * bx]; });
        }
        Real V[3];
        fluid_moments([&](auto qc) { return d[decltype(qc)::value]; }, drho, V);
        const Real rho = Real(1) + drho;
        const Real ie = rcp(eps);
        collide_tail<S, KMODE, SOLUTE>(
            a, n, g, [&](auto qc) { return d[decltype(qc)::value]; },
            [&](auto qc) { return src[(L::kH + decltype(qc)::value) * bx]; },
            [&](int k) { return src[(L::kKin + k) * bx]; }, drho, rho, V, ie, eps, sC, gx, gy, gz);
      } else {
        update_cell<S, KMODE, SOLUTE>(a, x, y, z, n, link, fin_acc, fout_acc, drho, sC, open_face);
      }
    }
    warp_reductions(a, warp_gid, open_face, fin_acc, fout_acc, drho, sC);
    s ^= 1u;
  }
  cp_async_wait<0>();
}

}  // namespace lbgb
