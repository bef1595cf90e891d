// Further solute species (species 1 .. S-1; species 0 is part of the fused
// step). Each species is a D3Q19 lattice of Eqs. equild / boltzeqD with its
// own tau_D and inlet concentration; all share the step's V' (and, at inlet
// faces, the bare streamed velocity V), which the fused step of the same
// step wrote to a.vel. The species pass runs after it, in the same launch
// shape, so each warp owns the same flux slots (offset per species).
//
// The arithmetic is the solute half of the per-cell update (update_cell and
// collide_tail in lb_kernels.cuh), written out here for one species at a
// time: the gather with its boundary classes, C = sum_q h_q / eps, h^eq at
// V* = V' + D_s grad(eps)/eps with the rest component as the remainder, BGK.
#pragma once

#include "lb_kernels.cuh"

namespace lbgb {

template <class S>
__device__ __forceinline__ void species_cell(const StepArgs<typename S::Real> &a, int sp,
                                             unsigned x, unsigned y, unsigned z, unsigned n,
                                             uint32_t link, typename S::Real &fin_acc,
                                             typename S::Real &fout_acc,
                                             typename S::Real &sC, bool &open_face) {
  using Real = typename S::Real;
  using T = typename S::T;
  const unsigned N = a.N;
  const CellGeo g = cell_geo_xyz(x, y, z, a.nx, a.ny, a.nz);
  // the paired layout keeps species 0 with f, so the h buffers start at species 1
  const size_t off = size_t(sp - a.paired) * Q * N;
  const T *__restrict__ hb = static_cast<const T *>(a.h_in) + off + n;
  T *__restrict__ ho = static_cast<T *>(a.h_out) + off + n;
  const float *rh_in = S::kShift ? a.rh_in + size_t(sp) * N : nullptr;
  const Real eps = __ldg(a.eps + n);
  const Real ratio = __ldg(a.spec + 16 + sp);  // D_s / D_0 (geps holds D_0 grad(eps)/eps)
  const Real gx = ratio * __ldg(a.geps + n), gy = ratio * __ldg(a.geps + N + n),
             gz = ratio * __ldg(a.geps + 2 * size_t(N) + n);
  const Real C_in = __ldg(a.spec + 8 + sp), itd = __ldg(a.spec + sp);
  const unsigned s_open = a.s_inlet | a.s_outlet;
  open_face = (g.onface & s_open) != 0;
  Real hh[Q];
  if (link == 0 && !(g.onface & (a.s_wall | s_open))) {
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      hh[q] = S::template ld_h<q>(hb + (int(q * N) + src_delta<q>(g)));
      if constexpr (S::kShift) hh[q] += wq<Real>(q) * __ldg(rh_in + (long long)n + src_delta<q>(g));
    });
  } else {
    const Real *vel = a.vel;
    const Real vi0 = __ldg(vel + n) + gx, vi1 = __ldg(vel + N + n) + gy,
               vi2 = __ldg(vel + 2 * size_t(N) + n) + gz;
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const int cls = solute_class<q>(g, link, a.s_wall, a.s_inlet, a.s_outlet);
      Real v;
      const Real own = S::kShift ? wq<Real>(q) * __ldg(rh_in + n) : Real(0);
      if (cls == PULL_CELL) {
        v = S::template ld_h<q>(hb + (int(q * N) + src_delta<q>(g)));
        if constexpr (S::kShift) v += wq<Real>(q) * __ldg(rh_in + (long long)n + src_delta<q>(g));
      } else if (cls == PULL_BOUNCE) {
        v = S::template ld_h<opp(q)>(hb + int(opp(q) * N)) + own;
      } else if (cls == PULL_INLET) {
        const Real cv = Real(cx(q)) * vi0 + Real(cy(q)) * vi1 + Real(cz(q)) * vi2;
        v = wq<Real>(q) * eps * C_in * (Real(1) + Real(3) * cv);
        fin_acc += v - (S::template ld_h<opp(q)>(hb + int(opp(q) * N)) + own);
      } else {
        v = S::template ld_h<q>(hb + int(q * N)) + own;
        fout_acc += (S::template ld_h<opp(q)>(hb + int(opp(q) * N)) + own) - v;
      }
      hh[q] = v;
    });
  }
  Unroll<0, Q>::run([&](auto qc) { sC += hh[decltype(qc)::value]; });
  const Real *vel = a.vel;
  const Real vs0 = __ldg(vel + 3 * size_t(N) + n) + gx, vs1 = __ldg(vel + 4 * size_t(N) + n) + gy,
             vs2 = __ldg(vel + 5 * size_t(N) + n) + gz;
  Real hsum = Real(0);
  Unroll<1, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const Real cv = Real(cx(q)) * vs0 + Real(cy(q)) * vs1 + Real(cz(q)) * vs2;
    const Real heq = wq<Real>(q) * sC * (Real(1) + Real(3) * cv);
    hsum += heq;
    const Real h = hh[q];
    const Real shift = S::kShift ? wq<Real>(q) * sC : Real(0);
    S::template st_h<q>(ho + int(q * N), h + (heq - h) * itd - shift);
  });
  {
    const Real h = hh[0];
    const Real shift = S::kShift ? wq<Real>(0) * sC : Real(0);
    S::template st_h<0>(ho, h + ((sC - hsum) - h) * itd - shift);
  }
  if constexpr (S::kShift) a.rh_out[size_t(sp) * N + n] = float(sC);
  if (a.fields) a.fields[(5 + size_t(sp)) * N + n] = float(sC * rcp(eps));
}

// Launch: the per-cell step kernel's shape (blocks of STEP_BLOCK threads, BX
// along x, grid (ceil(nx/BX), ceil(ny/BY), nz)).
template <class S>
__global__ void __launch_bounds__(STEP_BLOCK, 6) species_kernel(const StepArgs<typename S::Real> a) {
  using Real = typename S::Real;
  const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned y = blockIdx.y * blockDim.y + threadIdx.y;
  const unsigned z = blockIdx.z;
  const unsigned nx = a.nx, ny = a.ny;
  const unsigned warp_gid =
      ((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * (STEP_BLOCK / 32) +
      ((threadIdx.y * blockDim.x + threadIdx.x) >> 5);
  bool live = x < nx && y < ny;
  const unsigned n = x + nx * (y + ny * z);
  uint32_t link = 0;
  if (live && a.link) {
    link = __ldg(a.link + n);
    live = !(link >> 31);
  }
  const unsigned lane = threadIdx.x & 31u;  // blockDim.x is a multiple of 32
  for (int sp = 1; sp < a.species; ++sp) {
    Real fin_acc = Real(0), fout_acc = Real(0), sC = Real(0);
    bool open_face = false;
    if (live) species_cell<S>(a, sp, x, y, z, n, link, fin_acc, fout_acc, sC, open_face);
    // the per-warp reductions of the fused step, on this species' flux slots
    if (a.flux && __any_sync(0xffffffffu, open_face)) {
      const Real si = warp_sum(fin_acc), so = warp_sum(fout_acc);
      if (lane == 0) {
        double *slot = a.flux_slots + size_t(sp) * a.slot_stride + 2 * size_t(warp_gid);
        slot[0] += double(si);
        slot[1] += double(so);
      }
    }
    if (a.reduce) {
      const Real c = warp_sum(sC);
      if (lane == 0 && !isfinite(c)) atomicOr(&a.state->status, 1u);
    }
  }
}

// Initial species s >= 1 (flowchart step c), as the fused initialisation
// sets species 0: h = h^eq(eps, C0_s, u0 + D_s grad(eps)/eps) in both buffers
// (FP16/BF16: the reference is sum_q h^eq_q); solid cells 0.
template <class S>
__global__ void __launch_bounds__(BLOCK) species_init_kernel(const StepArgs<typename S::Real> a,
                                                             const float *u0, const float *C0) {
  using Real = typename S::Real;
  using T = typename S::T;
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  const unsigned N = a.N;
  if (n >= N) return;
  const bool solid = a.link && (__ldg(a.link + n) >> 31);
  const Real eps = a.eps[n];
  for (int sp = 1; sp < a.species; ++sp) {
    const size_t off = size_t(sp - a.paired) * Q * N;
    T *h0 = const_cast<T *>(static_cast<const T *>(a.h_in)) + off + n;
    T *h1 = static_cast<T *>(a.h_out) + off + n;
    const Real C = solid ? Real(0) : Real(C0[size_t(sp) * N + n]);
    const Real ratio = a.spec[16 + sp];
    const Real vs0 = Real(u0[3 * size_t(n)]) + ratio * a.geps[n];
    const Real vs1 = Real(u0[3 * size_t(n) + 1]) + ratio * a.geps[N + n];
    const Real vs2 = Real(u0[3 * size_t(n) + 2]) + ratio * a.geps[2 * size_t(N) + n];
    Real hs[Q];
    Real hsum = Real(0);
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const Real cv = Real(cx(q)) * vs0 + Real(cy(q)) * vs1 + Real(cz(q)) * vs2;
      hs[q] = solid ? Real(0) : wq<Real>(q) * eps * C * (Real(1) + Real(3) * cv);
      hsum += hs[q];
    });
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const Real h = hs[q] - (S::kShift ? wq<Real>(q) * hsum : Real(0));
      S::template st_h<q>(h0 + size_t(q) * N, h);
      S::template st_h<q>(h1 + size_t(q) * N, h);
    });
    if constexpr (S::kShift) {
      const_cast<float *>(a.rh_in)[size_t(sp) * N + n] = float(hsum);
      a.rh_out[size_t(sp) * N + n] = float(hsum);
    }
    if (a.fields) a.fields[(5 + size_t(sp)) * N + n] = solid ? 0.0f : float(C);
  }
}

}  // namespace lbgb
