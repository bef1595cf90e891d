// Instantiation of every per-cell kernel for one storage format; included by
// one small translation unit per format (lb_inst_*.cu).
#pragma once

#include "lb_free_surface.cuh"
#include "lb_kernels.cuh"
#include "lb_tma.cuh"
#include "lb_batch.cuh"
#include "lb_pipe.cuh"
#include "lb_species.cuh"
#include "lb_ops.h"

namespace lbgb {

// Calls f(km, sol) with the permeability mode and the solute setting as
// compile-time constants.
template <class F>
decltype(auto) dispatch_mode(int kmode, bool solute, F &&f) {
  using N = std::integral_constant<int, KM_NONE>;
  using D = std::integral_constant<int, KM_DIAG>;
  using P = std::integral_constant<int, KM_SPD>;
  using H = std::integral_constant<int, KM_FORCH>;
  using Y = std::true_type;
  using X = std::false_type;
  switch (kmode * 2 + (solute ? 1 : 0)) {
    case 0: return f(N{}, X{});
    case 1: return f(N{}, Y{});
    case 2: return f(D{}, X{});
    case 3: return f(D{}, Y{});
    case 4: return f(P{}, X{});
    case 5: return f(P{}, Y{});
    case 6: return f(H{}, X{});
    default: return f(H{}, Y{});
  }
}

template <class S>
struct Instance {
  using Real = typename S::Real;
  using A = StepArgs<Real>;

  template <int KM, bool SOL, int FEAT>
  static cudaError_t step_t(const A &a, dim3 grid, dim3 block, cudaStream_t s) {
    step_kernel<S, KM, SOL, FEAT><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t step(int kmode, bool solute, int feat, const void *args, dim3 grid,
                          dim3 block, cudaStream_t s) {
    const A &a = *static_cast<const A *>(args);
    return dispatch_mode(kmode, solute, [&](auto km, auto sol) {
      constexpr int K = decltype(km)::value;
      constexpr bool L = decltype(sol)::value;
      switch (feat) {
        case 0: return step_t<K, L, 0>(a, grid, block, s);
        case FEAT_OPEN: return step_t<K, L, FEAT_OPEN>(a, grid, block, s);
        case FEAT_SPEC: return L ? step_t<K, L, FEAT_SPEC>(a, grid, block, s) : cudaErrorInvalidValue;
        default:
          return L ? step_t<K, L, FEAT_OPEN | FEAT_SPEC>(a, grid, block, s) : cudaErrorInvalidValue;
      }
    });
  }
  static cudaError_t species_init(const void *args, const float *u0, const float *C0,
                                  unsigned nblk, cudaStream_t s) {
    species_init_kernel<S><<<nblk, BLOCK, 0, s>>>(*static_cast<const A *>(args), u0, C0);
    return cudaGetLastError();
  }
  template <int KM, bool SOL>
  static cudaError_t init_t(const A &a, const InitArgs<Real> &in, unsigned nblk, cudaStream_t s) {
    init_kernel<S, KM, SOL><<<nblk, BLOCK, 0, s>>>(a, in);
    return cudaGetLastError();
  }
  static cudaError_t init(int kmode, bool solute, const void *args, const void *init_args,
                          unsigned nblk, cudaStream_t s) {
    const A &a = *static_cast<const A *>(args);
    const InitArgs<Real> &in = *static_cast<const InitArgs<Real> *>(init_args);
    // the initial state does not depend on K; one instantiation per lattice set
    return solute ? init_t<KM_NONE, true>(a, in, nblk, s) : init_t<KM_NONE, false>(a, in, nblk, s);
  }
  static cudaError_t rhohat(const void *args, void *rh, unsigned nblk, cudaStream_t s) {
    rhohat_kernel<S><<<nblk, BLOCK, 0, s>>>(*static_cast<const A *>(args), static_cast<Real *>(rh));
    return cudaGetLastError();
  }
  // the references of FP32 / FP64 storage are ignored
  static PopView own_refs(PopView v) {
    if (!S::kShift) v.ref = nullptr;
    return v;
  }
  static cudaError_t to_f64(PopView src, double *dst, unsigned N, int lattice, cudaStream_t s) {
    const size_t tot = size_t(Q) * N;
    to_f64_kernel<S><<<unsigned((tot + BLOCK - 1) / BLOCK), BLOCK, 0, s>>>(own_refs(src), dst, N,
                                                                             lattice);
    return cudaGetLastError();
  }
  static cudaError_t from_f64(const double *src, PopView dst, unsigned N, int lattice,
                              cudaStream_t s) {
    const size_t tot = size_t(Q) * N;
    dst = own_refs(dst);
    if (S::kShift) ref_from_f64_kernel<<<(N + BLOCK - 1) / BLOCK, BLOCK, 0, s>>>(src, N, lattice, dst);
    from_f64_kernel<S><<<unsigned((tot + BLOCK - 1) / BLOCK), BLOCK, 0, s>>>(src, dst, N, lattice);
    return cudaGetLastError();
  }
  static cudaError_t totals(PopView f, PopView h, const uint32_t *link, unsigned N,
                            double *partials, unsigned nblk, cudaStream_t s) {
    totals_kernel<S><<<totals_blocks(nblk), BLOCK, 0, s>>>(own_refs(f), own_refs(h), link, N,
                                                          partials);
    return cudaGetLastError();
  }
  static cudaError_t fs_step(const void *args, unsigned grid, unsigned tile_blocks,
                             cudaStream_t s) {
    const FsArgs<Real> &f = *static_cast<const FsArgs<Real> *>(args);
    fs_mass_kernel<S><<<grid, FS_BLOCK, 0, s>>>(f);
    fs_step_kernel<S><<<grid, FS_BLOCK, 0, s>>>(f);
    fs_retype_kernel<Real><<<grid, FS_BLOCK, 0, s>>>(f);
    fs_newcell_kernel<S><<<grid, FS_BLOCK, 0, s>>>(f);
    fs_finish_kernel<S><<<grid, FS_BLOCK, 0, s>>>(f);
    (void)tile_blocks;
    return cudaGetLastError();
  }
  static cudaError_t fs_seed(const void *args, unsigned tiles, unsigned tile_blocks,
                             cudaStream_t s) {
    const FsArgs<Real> &f = *static_cast<const FsArgs<Real> *>(args);
    fs_seed_kernel<Real><<<tiles, FS_BLOCK, 0, s>>>(f);
    (void)tile_blocks;
    return cudaGetLastError();
  }
  // The row-pipelined kernel is built for the coupled lattice (solute on),
  // diagonal or full K, rows of 128 or 256 cells.
  template <int KM, int NW>
  static constexpr auto tma_kernel() {
    return &tma_step_kernel<S, KM, true, NW, (NW == 4 ? 3 : 2)>;
  }
  template <int KM, int NW>
  static bool tma_config_t(unsigned nx, size_t *smem, unsigned *threads, int *bps) {
    const size_t bytes = TmaLayout<S, KM, true>::smem_bytes(nx);
    int dev = 0, maxopt = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
    if (bytes > size_t(maxopt)) return false;
    if (cudaFuncSetAttribute(tma_kernel<KM, NW>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(bytes)) != cudaSuccess)
      return false;
    const unsigned thr = (NW + 1) * 32;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tma_kernel<KM, NW>(), int(thr), bytes) !=
            cudaSuccess ||
        nb < 1)
      return false;
    *smem = bytes;
    *threads = thr;
    *bps = nb;
    return true;
  }
  static bool tma_config(int kmode, bool solute, unsigned nx, size_t *smem, unsigned *threads,
                         int *bps) {
    if (!solute || kmode == KM_NONE || kmode == KM_FORCH || (nx != 128 && nx != 256))
      return false;
    if (kmode == KM_DIAG)
      return nx == 128 ? tma_config_t<KM_DIAG, 4>(nx, smem, threads, bps)
                       : tma_config_t<KM_DIAG, 8>(nx, smem, threads, bps);
    return nx == 128 ? tma_config_t<KM_SPD, 4>(nx, smem, threads, bps)
                     : tma_config_t<KM_SPD, 8>(nx, smem, threads, bps);
  }
  static cudaError_t tma_step(int kmode, bool solute, const void *args, unsigned grid,
                              unsigned threads, size_t smem, cudaStream_t s) {
    const A &a = *static_cast<const A *>(args);
    if (!solute || kmode == KM_NONE || kmode == KM_FORCH) return cudaErrorInvalidValue;
    const bool wide = threads == 9 * 32;
    if (kmode == KM_DIAG) {
      if (wide)
        tma_kernel<KM_DIAG, 8>()<<<grid, threads, smem, s>>>(a);
      else
        tma_kernel<KM_DIAG, 4>()<<<grid, threads, smem, s>>>(a);
    } else {
      if (wide)
        tma_kernel<KM_SPD, 8>()<<<grid, threads, smem, s>>>(a);
      else
        tma_kernel<KM_SPD, 4>()<<<grid, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
  }
  template <int KM, bool SOL>
  static bool pipe_config_t(unsigned bx, size_t *smem, int *bps) {
    const size_t bytes = PipeLayout<S, KM, SOL>::smem_bytes(bx);
    // the attribute is per kernel, shared by every context: always allow the
    // widest row, so that no context lowers it below another's launch
    const size_t widest = PipeLayout<S, KM, SOL>::smem_bytes(STEP_BLOCK);
    int dev = 0, maxopt = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
    if (widest > size_t(maxopt)) return false;
    if (cudaFuncSetAttribute(pipe_step_kernel<S, KM, SOL>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(widest)) != cudaSuccess)
      return false;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pipe_step_kernel<S, KM, SOL>, int(bx),
                                                      bytes) != cudaSuccess ||
        nb < 1)
      return false;
    *smem = bytes;
    *bps = nb;
    return true;
  }
  static bool pipe_config(int kmode, bool solute, unsigned bx, size_t *smem, int *bps) {
    if (bx != 32 && bx != 64 && bx != 128) return false;
    return dispatch_mode(kmode, solute, [&](auto km, auto sol) {
      return pipe_config_t<decltype(km)::value, decltype(sol)::value>(bx, smem, bps);
    });
  }
  static cudaError_t pipe_step(int kmode, bool solute, const void *args, unsigned grid,
                               unsigned bx, size_t smem, unsigned gxr, unsigned items,
                               cudaStream_t s) {
    const A &a = *static_cast<const A *>(args);
    dispatch_mode(kmode, solute, [&](auto km, auto sol) {
      pipe_step_kernel<S, decltype(km)::value, decltype(sol)::value><<<grid, bx, smem, s>>>(
          a, gxr, items);
    });
    return cudaGetLastError();
  }
  static cudaError_t batch_step(int kmode, bool solute, const void *tab, const uint64_t *work,
                                unsigned d_begin, unsigned vb_begin, unsigned vb_end,
                                unsigned grid, cudaStream_t s) {
    const BatchTable<Real> &t = *static_cast<const BatchTable<Real> *>(tab);
    dispatch_mode(kmode, solute, [&](auto km, auto sol) {
      batched_step_kernel<S, decltype(km)::value, decltype(sol)::value>
          <<<grid, STEP_BLOCK, 0, s>>>(t, work, d_begin, vb_begin, vb_end);
    });
    return cudaGetLastError();
  }
  static StorageOps make() {
    StorageOps o{};
    o.storage = S::id;
    o.elt_bytes = sizeof(typename S::T);
    o.fp64 = sizeof(Real) == 8;
    o.step = &step;
    o.init = &init;
    o.rhohat = &rhohat;
    o.to_f64 = &to_f64;
    o.from_f64 = &from_f64;
    o.totals = &totals;
    o.fs_step = nullptr;
    o.fs_seed = nullptr;
    if constexpr (S::id == StoreF32::id || S::id == StoreF64::id) {
      o.fs_step = &fs_step;
      o.fs_seed = &fs_seed;
    }
    o.batch_step = &batch_step;
    o.species_init = &species_init;
    o.tma_config = nullptr;
    o.tma_step = nullptr;
    o.pipe_config = nullptr;
    o.pipe_step = nullptr;
    if constexpr (sizeof(typename S::T) == sizeof(Real)) {  // FP32 and FP64 storage
      o.pipe_config = &pipe_config;
      o.pipe_step = &pipe_step;
    }
    if constexpr (S::id == StoreF32::id) {  // FP32 populations and static rows
      o.tma_config = &tma_config;
      o.tma_step = &tma_step;
    }
    return o;
  }
};

}  // namespace lbgb
