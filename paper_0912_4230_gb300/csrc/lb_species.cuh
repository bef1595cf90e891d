// Initial state of further solute species (species 1 .. S-1; species 0 is
// initialised with the fluid). Their steps are part of the per-cell step
// kernel (species_update in lb_kernels.cuh, kernel feature FEAT_SPEC).
#pragma once

#include "lb_kernels.cuh"

namespace lbgb {

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
