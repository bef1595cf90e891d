// Row-pipelined step kernel: the same per-cell update as step_kernel, with
// the populations and static fields of each x-row staged in shared memory by
// bulk asynchronous copies (cp.async.bulk, completed on mbarriers) so that
// HBM reads of the next rows overlap the collision of the current one.
//
// Persistent launch: gridDim.x blocks (a few per SM) walk the rows
// r = y + ny*z with stride gridDim.x. A block has nx/32 compute warps (one
// cell per thread, one x-row per tile) and one producer warp whose lane 0
// issues, for every tile, one bulk copy per source row: for each direction q
// the row (y - c_qy, z - c_qz) (wrapped on periodic faces) of f_q and h_q, and
// the cell's own rows of eps, K^-1 and D grad(eps)/eps. The x-shift of the
// pull is an index shift inside shared memory. Populations that do not come
// from a cell of a staged row (bounce-back, inlet, outlet) are read from
// global memory as in step_kernel.
//
// Every mbarrier wait is bounded; a wait that gives up sets bit 1 of the
// context status (reported as LB_ETIMEOUT) and the block stops.
#pragma once

#include "lb_kernels.cuh"

namespace lbgb {

constexpr int TMA_STAGES = 3;
// a wait gives up after this long (the global nanosecond timer), or after
// this many polls should the timer not advance
constexpr unsigned long long TMA_WAIT_NS = 1000000000ull;
constexpr unsigned TMA_WAIT_POLLS = 1u << 30;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: false when it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          unsigned long long limit_ns = TMA_WAIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned i = 0; i < TMA_WAIT_POLLS; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory layout of one stage, in units of rows of nx elements.
template <class S, int KMODE, bool SOLUTE>
struct TmaLayout {
  using T = typename S::T;
  static constexpr int kinv_rows = KMODE == KM_SPD ? 6 : (KMODE == KM_NONE ? 0 : 3);
  static constexpr int static_rows = 1 + kinv_rows + (SOLUTE ? 3 : 0);  // Real = float rows
  static constexpr int pop_rows = SOLUTE ? 2 * Q : Q;                    // T rows
  __host__ __device__ static size_t stage_bytes(unsigned nx) {
    return size_t(pop_rows) * nx * sizeof(T) + size_t(static_rows) * nx * sizeof(float);
  }
  __host__ __device__ static size_t smem_bytes(unsigned nx) {
    return 2 * TMA_STAGES * sizeof(uint64_t) + 16 + TMA_STAGES * stage_bytes(nx);
  }
};

// Shared-memory load that the compiler must not merge with an earlier load of
// the same address: the collision pass re-reads the staged populations
// instead of keeping all of them in registers.
template <class T>
__device__ __forceinline__ T lds_row(const T *p);
template <>
__device__ __forceinline__ float lds_row<float>(const float *p) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(smem_u32(p)));
  return v;
}
template <>
__device__ __forceinline__ __half lds_row<__half>(const __half *p) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(smem_u32(p)));
  return __ushort_as_half(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 lds_row<__nv_bfloat16>(const __nv_bfloat16 *p) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(smem_u32(p)));
  return __ushort_as_bfloat16(v);
}

// wrapped index shift of a pull source row: -1 when the row is behind a
// non-periodic face of the lattice (closed = wall | inlet | outlet faces)
__device__ __forceinline__ int source_row(int q, unsigned y, unsigned z, unsigned ny, unsigned nz,
                                          unsigned closed) {
  int ys = int(y) - cy(q), zs = int(z) - cz(q);
  if (ys < 0) {
    if (closed & 4u) return -1;
    ys += ny;
  } else if (ys >= int(ny)) {
    if (closed & 8u) return -1;
    ys -= ny;
  }
  if (zs < 0) {
    if (closed & 16u) return -1;
    zs += nz;
  } else if (zs >= int(nz)) {
    if (closed & 32u) return -1;
    zs -= nz;
  }
  return ys + int(ny) * zs;
}

// NW compute warps (nx = 32 NW) plus the producer warp; MINB resident blocks
// per SM bound the registers.
template <class S, int KMODE, bool SOLUTE, int NW, int MINB>
__global__ void __launch_bounds__(32 * (NW + 1), MINB)
    tma_step_kernel(const StepArgs<typename S::Real> a) {
  using Real = typename S::Real;
  using T = typename S::T;
  using L = TmaLayout<S, KMODE, SOLUTE>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);
  uint64_t *empty = full + TMA_STAGES;
  unsigned char *stage0 = smem + 2 * TMA_STAGES * sizeof(uint64_t) + 16;
  constexpr unsigned nx = 32 * NW;         // row length (the host launches only nx = 32 NW)
  const unsigned ny = a.ny, nz = a.nz, N = a.N;
  constexpr unsigned nwc = NW;             // compute warps
  const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const unsigned rows = ny * nz;
  const size_t sbytes = L::stage_bytes(nx);
  if (threadIdx.x == 0) {
    for (int s = 0; s < TMA_STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, nwc);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const unsigned my_tiles = blockIdx.x < rows ? (rows - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (warp == nwc) {
    // ---------------- producer ----------------
    if (lane != 0) return;
    const unsigned f_closed = a.f_wall;
    const unsigned s_closed = a.s_wall | a.s_inlet | a.s_outlet;
    const unsigned rowb = nx * sizeof(T), frowb = nx * sizeof(float);
    for (unsigned k = 0; k < my_tiles; ++k) {
      const unsigned s = k % TMA_STAGES;
      if (k >= TMA_STAGES && !mbar_wait(empty + s, ((k / TMA_STAGES) - 1) & 1u)) {
        atomicOr(&a.state->status, 2u);
        return;
      }
      const unsigned r = blockIdx.x + k * gridDim.x;
      const unsigned y = r % ny, z = r / ny;
      unsigned char *st = stage0 + s * sbytes;
      unsigned bytes = L::static_rows * frowb;
      for (int q = 0; q < Q; ++q) {
        if (source_row(q, y, z, ny, nz, f_closed) >= 0) bytes += rowb;
        if (SOLUTE && source_row(q, y, z, ny, nz, s_closed) >= 0) bytes += rowb;
      }
      mbar_arrive_expect_tx(full + s, bytes);
      const T *fin = static_cast<const T *>(a.f_in);
      for (int q = 0; q < Q; ++q) {
        const int fr = source_row(q, y, z, ny, nz, f_closed);
        if (fr >= 0)
          bulk_g2s(st + size_t(q) * rowb, fin + size_t(q) * N + size_t(fr) * nx, rowb, full + s);
      }
      if (SOLUTE) {
        const T *hin = static_cast<const T *>(a.h_in);
        for (int q = 0; q < Q; ++q) {
          const int hr = source_row(q, y, z, ny, nz, s_closed);
          if (hr >= 0)
            bulk_g2s(st + size_t(Q + q) * rowb, hin + size_t(q) * N + size_t(hr) * nx, rowb,
                     full + s);
        }
      }
      unsigned char *sf = st + size_t(L::pop_rows) * rowb;
      const size_t own = size_t(r) * nx;
      bulk_g2s(sf, a.eps + own, frowb, full + s);
      for (int k2 = 0; k2 < L::kinv_rows; ++k2)
        bulk_g2s(sf + size_t(1 + k2) * frowb, a.kinv + size_t(k2) * N + own, frowb, full + s);
      if (SOLUTE)
        for (int k2 = 0; k2 < 3; ++k2)
          bulk_g2s(sf + size_t(1 + L::kinv_rows + k2) * frowb, a.geps + size_t(k2) * N + own,
                   frowb, full + s);
    }
    // drain: wait until the consumers released the last stages, so no copy
    // into this block's shared memory is outstanding when it exits
    for (unsigned k = (my_tiles > TMA_STAGES ? my_tiles - TMA_STAGES : 0); k < my_tiles; ++k)
      if (!mbar_wait(empty + (k % TMA_STAGES), (k / TMA_STAGES) & 1u)) {
        atomicOr(&a.state->status, 2u);
        return;
      }
    return;
  }

  // ---------------- consumers ----------------
  const unsigned x = warp * 32 + lane;
  const unsigned warp_gid = blockIdx.x * nwc + warp;
  Real flux_in = Real(0), flux_out = Real(0);
  const unsigned rowb = nx * sizeof(T), frowb = nx * sizeof(float);
  for (unsigned k = 0; k < my_tiles; ++k) {
    const unsigned s = k % TMA_STAGES;
    // every lane waits (bounded), then the warp decides together, so a wait
    // that gives up never leaves part of a warp in the warp-wide reductions
    const bool ok = __all_sync(0xffffffffu, mbar_wait(full + s, (k / TMA_STAGES) & 1u));
    if (!ok) {
      if (lane == 0) atomicOr(&a.state->status, 2u);
      return;
    }
    const unsigned r = blockIdx.x + k * gridDim.x;
    const unsigned y = r % ny, z = r / ny;
    const unsigned n = x + nx * r;
    const unsigned char *st = stage0 + s * sbytes;
    const T *sfp = reinterpret_cast<const T *>(st);
    const T *shp = reinterpret_cast<const T *>(st + size_t(Q) * rowb);
    const float *sst = reinterpret_cast<const float *>(st + size_t(L::pop_rows) * rowb);
    uint32_t link = a.link ? __ldg(a.link + n) : 0u;
    const bool live = !(link >> 31);
    Real fa = Real(0), fo_ = Real(0), drho = Real(0), sC = Real(0);
    bool open_face = false;
    // a tile is interior when every pull source of every cell is a cell of a
    // staged row: no solid cell in the lattice, x periodic for both lattices,
    // and the row not on a non-periodic y or z face of either lattice
    const unsigned closed = a.f_wall | a.s_wall | a.s_inlet | a.s_outlet;
    const unsigned yzface = (y == 0 ? 4u : 0u) | (y == ny - 1 ? 8u : 0u) | (z == 0 ? 16u : 0u) |
                            (z == nz - 1 ? 32u : 0u);
    const bool interior = !a.link && !(closed & 3u) && !(yzface & closed);
    if (live && !interior) {
      update_cell<S, KMODE, SOLUTE>(a, x, y, z, n, link, fa, fo_, drho, sC, open_face);
    } else if (live) {
      const unsigned xm = (x == 0) ? nx - 1 : x - 1, xp = (x == nx - 1) ? 0 : x + 1;
      // arriving populations from the staged rows (re-read in the collision pass)
      auto fval = [&](auto qc) -> Real {
        constexpr int q = decltype(qc)::value;
        const unsigned xs = cx(q) > 0 ? xm : (cx(q) < 0 ? xp : x);
        return S::template cv_f<q>(lds_row<T>(sfp + q * nx + xs));
      };
      auto hval = [&](auto qc) -> Real {
        constexpr int q = decltype(qc)::value;
        const unsigned xs = cx(q) > 0 ? xm : (cx(q) < 0 ? xp : x);
        return S::template cv_h<q>(lds_row<T>(shp + q * nx + xs));
      };
      Real V[3];
      fluid_moments(fval, drho, V);
      const Real rho = Real(1) + drho;
      const Real eps = Real(sst[x]);
      const Real ie = rcp(eps);
      Real gx = Real(0), gy = Real(0), gz = Real(0);
      if (SOLUTE) {
        gx = Real(sst[(1 + L::kinv_rows) * nx + x]);
        gy = Real(sst[(2 + L::kinv_rows) * nx + x]);
        gz = Real(sst[(3 + L::kinv_rows) * nx + x]);
        Unroll<0, Q>::run([&](auto qc) { sC += hval(qc); });
      }
      // the collision pass re-reads the staged rows; K^-1 from shared memory
      collide_tail<S, KMODE, SOLUTE>(
          a, n, cell_geo_xyz(x, y, z, nx, ny, nz), fval, hval,
          [&](int k2) { return Real(sst[(1 + k2) * nx + x]); }, drho, rho, V, ie, eps, sC, gx, gy,
          gz);
    }
    // the stage may be refilled once every compute warp has read it
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + s);
    // reductions of this tile (whole warp participates)
    if (a.flux && __any_sync(0xffffffffu, open_face)) {
      flux_in += warp_sum(fa);
      flux_out += warp_sum(fo_);
    }
    if (a.reduce) {
      const Real m = warp_sum(drho), c = warp_sum(sC);
      if (lane == 0 && !(isfinite(m) && isfinite(c))) atomicOr(&a.state->status, 1u);
    }
  }
  if (a.flux && lane == 0 && (flux_in != Real(0) || flux_out != Real(0))) {
    a.flux_slots[2 * size_t(warp_gid)] += double(flux_in);
    a.flux_slots[2 * size_t(warp_gid) + 1] += double(flux_out);
  }
  (void)frowb;
}

}  // namespace lbgb
