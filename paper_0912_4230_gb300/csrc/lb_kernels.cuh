// Per-cell kernels of the GB300 lattice-Boltzmann library (templated on the
// population storage format, the permeability mode and the solute lattice).
//
// Layout: populations are structure-of-arrays, pop[q * N + n], n = x + nx*(y
// + ny*z), two buffers (A -> B -> A ...). Streaming is "pull": cell n reads
// f_q from n - c_q of the previous post-collision buffer, so every population
// is read once and written once per step and no atomics are needed. One
// thread owns one cell; consecutive threads are consecutive x, so each of the
// 19 loads and 19 stores of a warp is one contiguous 128-byte row segment
// (the x-shifted pulls straddle two segments, whose other half is read by the
// neighbouring warp and served from L1/L2).
#pragma once

#include <type_traits>

#include "lb_common.cuh"
#include "lb_ops.h"

namespace lbgb {

// Compile-time features of the per-cell step kernel, each a separate
// instantiation so that lattices without them keep the plain code:
// pressure / velocity faces of the fluid lattice, and further solute species
// (1 .. S-1, advanced by the same thread after the fluid and species 0).
enum : int { FEAT_OPEN = 1, FEAT_SPEC = 2 };

// the first direction of each pair of opposite directions (its partner is opp)
__host__ __device__ constexpr int pair_first(int k) {
  constexpr int t[9] = {1, 2, 5, 7, 8, 11, 13, 14, 17};
  return t[k];
}

template <int I, int N>
struct Unroll {
  template <class F>
  __device__ __forceinline__ static void run(F &&f) {
    f(std::integral_constant<int, I>{});
    Unroll<I + 1, N>::run(f);
  }
};
template <int N>
struct Unroll<N, N> {
  template <class F>
  __device__ __forceinline__ static void run(F &&) {}
};

template <class Real>
__device__ __forceinline__ Real warp_sum(Real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Geometry of one cell: wrapped index deltas to the six neighbours along the
// axes and the set of box faces the cell touches.
struct CellGeo {
  int dxm, dxp, dym, dyp, dzm, dzp;  // index delta to coord-1 / coord+1, wrapped
  unsigned onface;                   // faces_crossed bit layout
};

__device__ __forceinline__ CellGeo cell_geo_xyz(unsigned x, unsigned y, unsigned z, unsigned nx,
                                                unsigned ny, unsigned nz) {
  const int sy = int(nx), sz = int(nx * ny);
  CellGeo g;
  g.dxm = (x == 0) ? int(nx - 1) : -1;
  g.dxp = (x == nx - 1) ? -int(nx - 1) : 1;
  g.dym = (y == 0) ? int(ny - 1) * sy : -sy;
  g.dyp = (y == ny - 1) ? -int(ny - 1) * sy : sy;
  g.dzm = (z == 0) ? int(nz - 1) * sz : -sz;
  g.dzp = (z == nz - 1) ? -int(nz - 1) * sz : sz;
  g.onface = (x == 0 ? 1u : 0u) | (x == nx - 1 ? 2u : 0u) | (y == 0 ? 4u : 0u) |
             (y == ny - 1 ? 8u : 0u) | (z == 0 ? 16u : 0u) | (z == nz - 1 ? 32u : 0u);
  return g;
}

__device__ __forceinline__ CellGeo cell_geo(unsigned n, unsigned nx, unsigned ny, unsigned nz) {
  const unsigned x = n % nx, yz = n / nx, y = yz % ny, z = yz / ny;
  return cell_geo_xyz(x, y, z, nx, ny, nz);
}

// index delta of the pull source n - c_q (wrapped)
template <int q>
__device__ __forceinline__ int src_delta(const CellGeo &g) {
  return (cx(q) > 0 ? g.dxm : (cx(q) < 0 ? g.dxp : 0)) +
         (cy(q) > 0 ? g.dym : (cy(q) < 0 ? g.dyp : 0)) +
         (cz(q) > 0 ? g.dzm : (cz(q) < 0 ? g.dzp : 0));
}
// index delta of the neighbour n + c_q (wrapped)
template <int q>
__device__ __forceinline__ int ahead_delta(const CellGeo &g) {
  return src_delta<opp(q)>(g);
}

// Pull classes (shared by the step kernels and the debug export, which
// reports class c as -(1 + c)).
enum : int { PULL_CELL = 0, PULL_BOUNCE = 1, PULL_INLET = 2, PULL_OUTLET = 3,
             PULL_PRESSURE = 5, PULL_VELOCITY = 6 };

// Fluid class of population q: across a wall face or from a solid cell
// bounce-back; across a velocity face, else a pressure face, that face's
// rule (walls take precedence on edges, then velocity, then pressure).
template <int q>
__device__ __forceinline__ int fluid_class(const CellGeo &g, uint32_t link, unsigned f_wall) {
  if (q == 0) return PULL_CELL;
  const unsigned fc = faces_crossed(q) & g.onface;
  if (fc & f_wall) return PULL_BOUNCE;
  return ((link >> q) & 1u) ? PULL_BOUNCE : PULL_CELL;
}
template <int q>
__device__ __forceinline__ int fluid_class_open(const CellGeo &g, uint32_t link, unsigned f_wall,
                                                unsigned f_vel, unsigned f_press) {
  const unsigned fc = faces_crossed(q) & g.onface;
  if (q != 0 && !(fc & f_wall)) {
    if (fc & f_vel) return PULL_VELOCITY;
    if (fc & f_press) return PULL_PRESSURE;
  }
  return fluid_class<q>(g, link, f_wall);
}
// the face (2 axis + side) of kind `mask` that population q crosses first in
// axis order
template <int q>
__device__ __forceinline__ int crossed_face(const CellGeo &g, unsigned mask) {
  return __ffs(faces_crossed(q) & g.onface & mask) - 1;
}

template <int q>
__device__ __forceinline__ int solute_class(const CellGeo &g, uint32_t link, unsigned s_wall,
                                            unsigned s_inlet, unsigned s_outlet) {
  if (q == 0) return PULL_CELL;
  const unsigned fc = faces_crossed(q) & g.onface;
  if (fc & s_wall) return PULL_BOUNCE;
  if (fc & s_inlet) return PULL_INLET;
  if (fc & s_outlet) return PULL_OUTLET;
  return ((link >> q) & 1u) ? PULL_BOUNCE : PULL_CELL;
}

// Stream the fluid populations into d[] (f_q - w_q of the arriving populations).
// paired: 16-bit storage in the paired layout (rf then holds __half2 pairs).
template <class S>
__device__ __forceinline__ void gather_f(const typename S::T *__restrict__ fin, unsigned N,
                                         unsigned n, const CellGeo &g, uint32_t link,
                                         unsigned f_wall, typename S::Real (&d)[Q],
                                         const float *rf = nullptr, bool paired = false) {
  using Real = typename S::Real;
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int cls = fluid_class<q>(g, link, f_wall);
    const long long src = (cls == PULL_BOUNCE) ? (long long)n : (long long)n + src_delta<q>(g);
    const size_t idx = (cls == PULL_BOUNCE) ? size_t(opp(q)) * N + n : size_t(q) * N + src;
    if constexpr (S::kShift) {
      if (paired)
        d[q] = wq<Real>(q) * (S::ld2(reinterpret_cast<const typename S::T2 *>(fin) + idx).x +
                              ld_ref2(rf + src).x);
      else
        d[q] = S::template ld_f<q>(fin + idx) + wq<Real>(q) * __ldg(rf + src);
    } else {
      d[q] = S::template ld_f<q>(fin + idx);
    }
  });
}

// Relaxation time from the viscosity law (Section 2, after Eq. eqsurftens;
// Eq. nuall for law 2 with t the step index after the increment).
template <class Real>
__device__ __forceinline__ Real tau_of(const StepArgs<Real> &a, Real C) {
  if (a.visc_law == 1) {
    const Real cl = C < Real(0) ? Real(0) : (C > Real(1) ? Real(1) : C);
    return a.tau0 + (a.tau1 - a.tau0) * cl;
  }
  if (a.visc_law == 2) {
    const Real nu = a.nu_g * (Real(1) + a.a_h * exp(a.alpha * Real(a.t))) *
                    exp(a.beta * (Real(1) - C));
    return Real(3) * nu + Real(0.5);
  }
  return a.tau;
}

// Reciprocal in the collision type: one correctly rounded reciprocal
// instruction sequence in FP32, exact division in FP64.
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// Inside an iteration that corrects its own errors (the Forchheimer Newton
// solve) FP32 takes the hardware's single-instruction approximations (at
// most 1 ulp off: PTX rcp.approx / sqrt.approx); FP64 keeps exact operations.
__device__ __forceinline__ float rcp_iter(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double rcp_iter(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_iter(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double sqrt_iter(double x) { return sqrt(x); }

// V' = Lambda^-1 (V + eps G / 2), Lambda = I + (eps nu / 2) K^-1, and
// F^ext = -eps nu K^-1 V' + eps G (Eqs. forcement, expandV, expandVsub).
// kv(r) returns row r of the cell's K^-1 (diagonal: xx, yy, zz; full: xx, yy,
// zz, xy, yz, zx).
//
// KM_FORCH adds the Forchheimer drag of the porous-flow model the paper builds
// on (the paper names the term without an equation): F^ext = -eps nu K^-1 V'
// - eps F_eps |V'| K^-1/2 V' + eps G, F_eps = cF 1.75 / sqrt(150 eps^3), for a
// diagonal K. With V' = V + F^ext/2, V'_i = r_i / (a_i + b_i s), r = V + eps
// G/2, a_i = 1 + eps nu k_i / 2, b_i = eps F_eps sqrt(k_i) / 2, where s = |V'|
// is the root of phi(s) = s - |V'(s)|. Newton's method on phi from the
// closed form of an isotropic medium with the r^2-weighted a and b; three
// iterations in FP32 and four in FP64 reach the root to rounding for K from
// 1e-4 to 1e2, 100:1 anisotropy and cF up to 20.
template <int KMODE, class Real, class KV>
__device__ __forceinline__ void velocity_solve_kv(KV kv, Real eps, Real nu, const Real (&V)[3],
                                                  const Real (&G)[3], Real cF, Real (&Vp)[3],
                                                  Real (&Fe)[3]) {
  const Real r0 = V[0] + Real(0.5) * eps * G[0];
  const Real r1 = V[1] + Real(0.5) * eps * G[1];
  const Real r2 = V[2] + Real(0.5) * eps * G[2];
  const Real en = eps * nu;
  if (KMODE == KM_NONE) {
    Vp[0] = r0; Vp[1] = r1; Vp[2] = r2;
    Fe[0] = eps * G[0]; Fe[1] = eps * G[1]; Fe[2] = eps * G[2];
  } else if (KMODE == KM_FORCH) {
    const Real k[3] = {kv(0), kv(1), kv(2)};
    const Real r[3] = {r0, r1, r2};
    const Real Fer = cF * Real(1.75) * rcp(sqrt(Real(150) * eps * eps * eps));
    const Real hs = Real(0.5) * en, hc = Real(0.5) * eps * Fer;
    Real a[3], b[3], d[3];
    for (int i = 0; i < 3; ++i) {
      d[i] = sqrt(k[i]);
      a[i] = Real(1) + hs * k[i];
      b[i] = hc * d[i];
    }
    const Real ws = r0 * r0 + r1 * r1 + r2 * r2;
    Real s = Real(0);
    if (ws > Real(0)) {
      const Real iws = rcp(ws);
      const Real ab = (r0 * r0 * a[0] + r1 * r1 * a[1] + r2 * r2 * a[2]) * iws;
      const Real bb = (r0 * r0 * b[0] + r1 * r1 * b[1] + r2 * r2 * b[2]) * iws;
      const Real rn = sqrt(ws);
      s = Real(2) * rn * rcp_iter(ab + sqrt_iter(ab * ab + Real(4) * bb * rn));
      // Newton on phi(s) = s - |V'(s)|: s <- s - (s - |V'|) |V'| / (|V'| + g),
      // g = sum_i V'_i^2 b_i / (a_i + b_i s); the iteration absorbs the
      // approximate reciprocals and roots, the final V' takes exact ones
      constexpr int kIters = sizeof(Real) == 4 ? 3 : 4;
      for (int it = 0; it < kIters; ++it) {
        Real vv = Real(0), g = Real(0);
        for (int i = 0; i < 3; ++i) {
          const Real iD = rcp_iter(a[i] + b[i] * s), v = r[i] * iD;
          vv += v * v;
          g += v * v * b[i] * iD;
        }
        const Real vn = sqrt_iter(vv);
        s -= (s - vn) * vn * rcp_iter(vn + g);
      }
    }
    for (int i = 0; i < 3; ++i) Vp[i] = r[i] * rcp(a[i] + b[i] * s);
    const Real sp = sqrt(Vp[0] * Vp[0] + Vp[1] * Vp[1] + Vp[2] * Vp[2]);
    for (int i = 0; i < 3; ++i) Fe[i] = -(en * k[i] + eps * Fer * d[i] * sp) * Vp[i] + eps * G[i];
  } else if (KMODE == KM_DIAG) {
    const Real kx = kv(0), ky = kv(1), kz = kv(2);
    const Real hs = Real(0.5) * en;
    Vp[0] = r0 * rcp(Real(1) + hs * kx);
    Vp[1] = r1 * rcp(Real(1) + hs * ky);
    Vp[2] = r2 * rcp(Real(1) + hs * kz);
    Fe[0] = -en * kx * Vp[0] + eps * G[0];
    Fe[1] = -en * ky * Vp[1] + eps * G[1];
    Fe[2] = -en * kz * Vp[2] + eps * G[2];
  } else {
    const Real kxx = kv(0), kyy = kv(1), kzz = kv(2);
    const Real kxy = kv(3), kyz = kv(4), kzx = kv(5);
    const Real hs = Real(0.5) * en;
    const Real l00 = Real(1) + hs * kxx, l11 = Real(1) + hs * kyy, l22 = Real(1) + hs * kzz;
    const Real l01 = hs * kxy, l12 = hs * kyz, l02 = hs * kzx;
    // adjugate of the symmetric matrix Lambda
    const Real c00 = l11 * l22 - l12 * l12, c01 = l02 * l12 - l01 * l22, c02 = l01 * l12 - l02 * l11;
    const Real c11 = l00 * l22 - l02 * l02, c12 = l01 * l02 - l00 * l12, c22 = l00 * l11 - l01 * l01;
    const Real idet = Real(1) / (l00 * c00 + l01 * c01 + l02 * c02);
    Vp[0] = (c00 * r0 + c01 * r1 + c02 * r2) * idet;
    Vp[1] = (c01 * r0 + c11 * r1 + c12 * r2) * idet;
    Vp[2] = (c02 * r0 + c12 * r1 + c22 * r2) * idet;
    Fe[0] = -en * (kxx * Vp[0] + kxy * Vp[1] + kzx * Vp[2]) + eps * G[0];
    Fe[1] = -en * (kxy * Vp[0] + kyy * Vp[1] + kyz * Vp[2]) + eps * G[1];
    Fe[2] = -en * (kzx * Vp[0] + kyz * Vp[1] + kzz * Vp[2]) + eps * G[2];
  }
}

template <int KMODE, class Real>
__device__ __forceinline__ void velocity_solve(const Real *__restrict__ kinv, unsigned N,
                                               unsigned n, Real eps, Real nu, const Real (&V)[3],
                                               const Real (&G)[3], Real (&Vp)[3],
                                               Real (&Fe)[3]) {
  velocity_solve_kv<KMODE>([&](int r) { return __ldg(kinv + size_t(r) * N + n); }, eps, nu, V, G,
                           Real(0), Vp, Fe);
}

// Colour gradient F = sum_q rhohat(x + c_q) c_q (Eq. macros); a step out
// through a wall face sees wall_rho (solid cells already hold wall_rho).
template <class Real>
__device__ __forceinline__ void colour_gradient(const Real *__restrict__ rh, unsigned n,
                                                const CellGeo &g, unsigned f_wall, Real wall_rho,
                                                Real (&F)[3]) {
  F[0] = F[1] = F[2] = Real(0);
  Unroll<1, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const bool out = (faces_ahead(q) & g.onface & f_wall) != 0;
    const Real r = out ? wall_rho : __ldg(rh + (long long)n + ahead_delta<q>(g));
    if (cx(q)) F[0] += Real(cx(q)) * r;
    if (cy(q)) F[1] += Real(cy(q)) * r;
    if (cz(q)) F[2] += Real(cz(q)) * r;
  });
}

// BGK collision with the porous equilibrium (Eqs. equilc1, equilc2) and the
// forcing terms (Eq. coeffforce1, with the weight and density factor w_q rho)
// for one direction, in deviation form:
//   f~_q - w_q = (f_q - w_q)(1 - 1/tau) + (f^eq_q - w_q)/tau + T_q.
// fold() gathers the per-cell factors of the last two terms, so that per
// direction they are w_q b_q with
//   b_q = K + cu (B3 + B45 cu + P9 cF) + P3 cF [+ S2 (c_q.F)^2],
// cu = c_q.V', cF = c_q.F_e (K0 in place of K for the rest direction), taken
// as scale (b_q - shift): scale 1 and shift 0 give the deviation above;
// 16-bit storage folds its scale and the cell's reference into them.
template <class Real>
struct FluidCollide {
  Real drho, rho, ie, uu, uF, itau, omt, pre, stc, Fn, iFn;
  Real Vp[3], Fe[3], F[3];
  bool st;
  Real K, K0, B3, B45, P9, P3, S2;

  __device__ __forceinline__ void fold(Real scale, Real shift) {
    // 1/tau (f^eq - w) + T at cu = cF = 0, without the surface-tension part
    const Real kb = itau * drho - Real(1.5) * itau * rho * ie * uu - Real(3) * pre * ie * uF;
    const Real ks = st ? itau * stc * Fn : Real(0);
    K = scale * (kb - ks - shift);
    K0 = scale * (kb + ks - shift);
    B3 = scale * Real(3) * itau * rho;
    B45 = scale * Real(4.5) * itau * rho * ie;
    P9 = scale * Real(9) * pre * ie;
    P3 = scale * Real(3) * pre;
    S2 = st ? scale * itau * stc * iFn : Real(0);
  }
  template <int q>
  __device__ __forceinline__ Real br() const {
    if (q == 0) return K0;
    const Real cu = Real(cx(q)) * Vp[0] + Real(cy(q)) * Vp[1] + Real(cz(q)) * Vp[2];
    const Real cF = Real(cx(q)) * Fe[0] + Real(cy(q)) * Fe[1] + Real(cz(q)) * Fe[2];
    Real b = cu * (B3 + B45 * cu + P9 * cF) + (P3 * cF + K);
    if (st) {
      const Real cs = Real(cx(q)) * F[0] + Real(cy(q)) * F[1] + Real(cz(q)) * F[2];
      b += S2 * cs * cs;
    }
    return b;
  }
  // b_q and b_qbar of a pair of opposite directions: the even part K +
  // cu (B45 cu + P9 cF) [+ S2 (c.F)^2] is shared, the odd part B3 cu + P3 cF
  // changes sign (cu = c_q.V', cF = c_q.F_e). Every step is an explicit
  // fma, product or sum, so every kernel rounds it alike.
  template <int q>
  __device__ __forceinline__ void br_pair(Real &bq, Real &bo) const {
    const Real cu = Real(cx(q)) * Vp[0] + Real(cy(q)) * Vp[1] + Real(cz(q)) * Vp[2];
    const Real cF = Real(cx(q)) * Fe[0] + Real(cy(q)) * Fe[1] + Real(cz(q)) * Fe[2];
    Real ev = fma(cu, fma(B45, cu, P9 * cF), K);
    if (st) {
      const Real cs = Real(cx(q)) * F[0] + Real(cy(q)) * F[1] + Real(cz(q)) * F[2];
      ev = fma(S2 * cs, cs, ev);
    }
    const Real od = fma(B3, cu, P3 * cF);
    bq = ev + od;
    bo = ev - od;
  }
  // f^eq_q - w_q (with the surface-tension part), for initialisation
  template <int q>
  __device__ __forceinline__ Real feq_dev() const {
    constexpr Real w = wq<Real>(q);
    if (q == 0) return w * (drho - rho * Real(1.5) * ie * uu) + (st ? stc * w * Fn : Real(0));
    const Real cu = Real(cx(q)) * Vp[0] + Real(cy(q)) * Vp[1] + Real(cz(q)) * Vp[2];
    Real e = w * (drho + rho * (Real(3) * cu + Real(4.5) * ie * cu * cu - Real(1.5) * ie * uu));
    if (st) {
      const Real cs = Real(cx(q)) * F[0] + Real(cy(q)) * F[1] + Real(cz(q)) * F[2];
      e += w * stc * (cs * cs * iFn - Fn);
    }
    return e;
  }
  // f~_q - w_q after fold(1, 0)
  template <int q>
  __device__ __forceinline__ Real post(Real d) const {
    return fma(wq<Real>(q), br<q>(), d * omt);
  }
};

// Exported fields, 6 x N floats: rho [N], u packed per cell [3N], C [N], nu [N].
template <class Real>
__device__ __forceinline__ void write_fields(float *fl, unsigned N, unsigned n, Real rho,
                                             const Real (&u)[3], Real C, Real nu) {
  fl[n] = float(rho);
  fl[size_t(N) + 3 * size_t(n)] = float(u[0]);
  fl[size_t(N) + 3 * size_t(n) + 1] = float(u[1]);
  fl[size_t(N) + 3 * size_t(n) + 2] = float(u[2]);
  fl[4 * size_t(N) + n] = float(C);
  fl[5 * size_t(N) + n] = float(nu);
}

__device__ __forceinline__ void zero_fields(float *fl, unsigned N, unsigned n) {
  fl[n] = 0.0f;
  fl[size_t(N) + 3 * size_t(n)] = 0.0f;
  fl[size_t(N) + 3 * size_t(n) + 1] = 0.0f;
  fl[size_t(N) + 3 * size_t(n) + 2] = 0.0f;
  fl[4 * size_t(N) + n] = 0.0f;
  fl[5 * size_t(N) + n] = 0.0f;
}

template <class Real>
__device__ __forceinline__ Real st_threshold();
template <>
__device__ __forceinline__ float st_threshold<float>() { return 1e-20f; }
template <>
__device__ __forceinline__ double st_threshold<double>() { return 1e-30; }

// Per-warp FP64 reductions of a step. Solute fluxes through inlet/outlet
// faces are accumulated into one FP64 slot pair per warp of the launch
// (each warp owns its slots across steps, so the running sums are
// deterministic; lb_reduce adds the slots in a fixed order). On checked
// steps the warp's mass and solute sums are tested for NaN/Inf.
template <class Real>
__device__ __forceinline__ void warp_reductions(const StepArgs<Real> &a, unsigned warp_gid,
                                                bool open_face, Real fin, Real fout, Real drho,
                                                Real sC) {
  const unsigned lane = threadIdx.x & 31u;
  if (a.flux && __any_sync(0xffffffffu, open_face)) {
    const Real si = warp_sum(fin), so = warp_sum(fout);
    if (lane == 0) {
      a.flux_slots[2 * size_t(warp_gid)] += double(si);
      a.flux_slots[2 * size_t(warp_gid) + 1] += double(so);
    }
  }
  if (a.reduce) {
    const Real m = warp_sum(drho), c = warp_sum(sC);
    if (lane == 0 && !(isfinite(m) && isfinite(c))) atomicOr(&a.state->status, 1u);
  }
}

// Stream of a cell on a pressure or velocity face of the fluid lattice into
// d[] (f_q - w_q). The face rules need the cell's own post-collision density
// and velocity, from its 19 populations of the input buffer: a population
// entering through a pressure face is -f~_qbar + 2 w_q rho_b (1 + 4.5
// (c_q.u)^2/eps - 1.5 u.u/eps) with rho_b = 3 eps P_face; through a velocity
// face f~_qbar + 6 w_q rho (c_q . u_face). Kept out of line: face cells are
// few, and the hot path keeps its registers.
template <class Real>
struct Pops {
  Real v[Q];
};

template <class S>
__device__ __noinline__ Pops<typename S::Real> gather_open_faces(
    const StepArgs<typename S::Real> &a, const CellGeo &g, unsigned n, uint32_t link) {
  using Real = typename S::Real;
  Pops<Real> d;
  using T = typename S::T;
  const unsigned N = a.N;
  const T *__restrict__ fb = static_cast<const T *>(a.f_in) + n;
  Real own[Q];
  Real r = Real(0), j0 = Real(0), j1 = Real(0), j2 = Real(0);
  // 16-bit storage: f_q - w_q = w_q (remainder + reference), from the pairs
  // of the paired layout or the plain rows
  auto ld_src = [&](auto qc, int off, int roff) -> Real {
    constexpr int q = decltype(qc)::value;
    if constexpr (S::kShift) {
      if (a.paired)
        return wq<Real>(q) * (S::ld2(static_cast<const typename S::T2 *>(a.f_in) + n + off).x +
                              ld_ref2(a.rf_in + (long long)n + roff).x);
      return S::template ld_f<q>(fb + off) + wq<Real>(q) * __ldg(a.rf_in + (long long)n + roff);
    } else {
      return S::template ld_f<q>(fb + off);
    }
  };
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const Real v = ld_src(qc, int(q * N), 0);
    own[q] = v;
    r += v;
    if (cx(q)) j0 += Real(cx(q)) * v;
    if (cy(q)) j1 += Real(cy(q)) * v;
    if (cz(q)) j2 += Real(cz(q)) * v;
  });
  const Real rho = Real(1) + r, irho = rcp(rho);
  const Real u0 = j0 * irho, u1 = j1 * irho, u2 = j2 * irho;
  const Real ie = rcp(__ldg(a.eps + n)), eps = __ldg(a.eps + n);
  const Real uu = u0 * u0 + u1 * u1 + u2 * u2;
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int cls = fluid_class_open<q>(g, link, a.f_wall, a.f_vel, a.f_press);
    Real v;
    if (cls == PULL_BOUNCE) {
      v = own[opp(q)];
    } else if (cls == PULL_PRESSURE) {
      // rho_b - 1 from 3P = hi + lo with one rounding of eps hi - 1
      const int fi = crossed_face<q>(g, a.f_press);
      const Real rbm1 = fma(eps, __ldg(a.face + fi), Real(-1)) + eps * __ldg(a.face + 24 + fi);
      const Real rb = Real(1) + rbm1;
      const Real cu = Real(cx(q)) * u0 + Real(cy(q)) * u1 + Real(cz(q)) * u2;
      const Real e = wq<Real>(q) * (rbm1 + rb * (Real(4.5) * ie * cu * cu - Real(1.5) * ie * uu));
      v = Real(2) * e - own[opp(q)];
    } else if (cls == PULL_VELOCITY) {
      const Real *uf = a.face + 6 + 3 * crossed_face<q>(g, a.f_vel);
      const Real cub = Real(cx(q)) * __ldg(uf) + Real(cy(q)) * __ldg(uf + 1) +
                       Real(cz(q)) * __ldg(uf + 2);
      v = own[opp(q)] + Real(6) * wq<Real>(q) * rho * cub;
    } else {
      v = ld_src(qc, int(q * N) + src_delta<q>(g), src_delta<q>(g));
    }
    d.v[q] = v;
  });
  return d;
}

// Fluid moments of the arriving populations: drho += sum_q (f_q - w_q) and
// V = j / rho with j = sum_q c_q (f_q - w_q), rho = 1 + drho. With E the
// values are e_q = (f_q - w_q)/w_q (16-bit storage) and carry their weights
// here.
template <bool E = false, class Real, class FV>
__device__ __forceinline__ void fluid_moments(FV fv, Real &drho, Real (&V)[3]) {
  Real j0 = Real(0), j1 = Real(0), j2 = Real(0);
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const Real v = fv(qc);
    if constexpr (E) {
      constexpr Real w = wq<Real>(q);
      drho = fma(w, v, drho);
      if (cx(q)) j0 = fma(Real(cx(q)) * w, v, j0);
      if (cy(q)) j1 = fma(Real(cy(q)) * w, v, j1);
      if (cz(q)) j2 = fma(Real(cz(q)) * w, v, j2);
    } else {
      drho += v;
      if (cx(q)) j0 += Real(cx(q)) * v;
      if (cy(q)) j1 += Real(cy(q)) * v;
      if (cz(q)) j2 += Real(cz(q)) * v;
    }
  });
  const Real irho = rcp(Real(1) + drho);
  V[0] = j0 * irho;
  V[1] = j1 * irho;
  V[2] = j2 * irho;
}

// The per-cell arithmetic after streaming: concentration and viscosity,
// colour gradient, V' and the Darcy force, fluid and solute collision,
// stores and exported fields. fv(q) and hv(q) give the arriving f_q - w_q and
// h_q (16-bit storage: (f_q - w_q)/w_q and h_q/w_q), kv(r) the rows of K^-1;
// drho, rho, V are the fluid moments, sC the solute total of the arriving h.
// VOUT: the cell's bare V and V' are returned in vout[0..2], vout[3..5]
// (for the further solute species of the same thread).
template <class S, int KMODE, bool SOLUTE, bool VOUT = false, class FV, class HV, class KV>
__device__ __forceinline__ void collide_tail(const StepArgs<typename S::Real> &a, unsigned n,
                                             const CellGeo &g, FV fv, HV hv, KV kv,
                                             typename S::Real drho, typename S::Real rho,
                                             const typename S::Real (&V)[3], typename S::Real ie,
                                             typename S::Real eps, typename S::Real sC,
                                             typename S::Real gx, typename S::Real gy,
                                             typename S::Real gz,
                                             typename S::Real *vout = nullptr) {
  using Real = typename S::Real;
  using T = typename S::T;
  const unsigned N = a.N;
  T *__restrict__ fo = static_cast<T *>(a.f_out) + n;
  const Real C = sC * ie;
  const Real tau = tau_of(a, C);
  const Real nu = (tau - Real(0.5)) * Real(1.0 / 3.0);

  FluidCollide<Real> fc;
  fc.F[0] = fc.F[1] = fc.F[2] = Real(0);
  if (a.A != Real(0)) colour_gradient(a.rhohat, n, g, a.f_wall, a.wall_rho, fc.F);
  velocity_solve_kv<KMODE>(kv, eps, nu, V, a.G, a.forch, fc.Vp, fc.Fe);
  fc.drho = drho;
  fc.rho = rho;
  fc.ie = ie;
  fc.uu = fc.Vp[0] * fc.Vp[0] + fc.Vp[1] * fc.Vp[1] + fc.Vp[2] * fc.Vp[2];
  fc.uF = fc.Vp[0] * fc.Fe[0] + fc.Vp[1] * fc.Fe[1] + fc.Vp[2] * fc.Fe[2];
  fc.itau = rcp(tau);
  fc.omt = Real(1) - fc.itau;
  fc.pre = rho * (Real(1) - Real(0.5) * fc.itau);
  fc.st = false;
  fc.Fn = fc.stc = fc.iFn = Real(0);
  if (a.A != Real(0)) {
    fc.Fn = sqrt(fc.F[0] * fc.F[0] + fc.F[1] * fc.F[1] + fc.F[2] * fc.F[2]);
    fc.st = fc.Fn > st_threshold<Real>();
    fc.stc = fc.st ? a.A * eps * tau : Real(0);
    fc.iFn = fc.st ? Real(1) / fc.Fn : Real(0);
  }
  if constexpr (S::kShift && SOLUTE) {
    // paired layout: both lattices per unit weight in one loop, one 32-bit
    // pair store per direction. The references are drho and sC rounded to
    // FP16; the remainders are formed against the rounded values.
    // f: (f~_q - w_q)/w_q = omt e_q + b_q, stored scale ((f~_q - w_q)/w_q - Rf).
    // h: h~_q/w_q = (1 - 1/tau_D) h_q/w_q + h^eq_q/(w_q tau_D) with
    // h^eq_q/w_q = sC (1 + 3 c_q.v), stored scale (h~_q/w_q - Rh); the rest
    // direction takes sC - sum_{q>0} h^eq_q, divided by its weight with a
    // correctly rounded division, so the weights' rounding adds no solute.
    // Opposite directions are formed together: they share c.V', c.F_e and
    // c.v, and their h^eq sum to 2 w sC.
    const __half2 r2 = __floats2half2_rn(drho, sC);
    const float2 R = __half22float2(r2);
    using T2 = typename S::T2;
    T2 *__restrict__ po = static_cast<T2 *>(a.f_out) + n;
    const Real sc = Real(S::kScale);
    fc.fold(sc, R.x);
    const Real so = sc * fc.omt;
    const Real vs0 = fc.Vp[0] + gx, vs1 = fc.Vp[1] + gy, vs2 = fc.Vp[2] + gz;
    const Real itd = a.inv_tau_D;
    const Real sod = sc * (Real(1) - itd), h0 = sc * (itd * sC - R.y),
               h3 = Real(3) * sc * itd * sC;
    Real hsum = Real(0);
    Unroll<0, 9>::run([&](auto kc) {
      constexpr int q = pair_first(decltype(kc)::value), o = opp(q);
      const auto qq = std::integral_constant<int, q>{};
      const auto oo = std::integral_constant<int, o>{};
      const Real cv = Real(cx(q)) * vs0 + Real(cy(q)) * vs1 + Real(cz(q)) * vs2;
      hsum = fma(Real(2) * wq<Real>(q), sC, hsum);
      Real bq, bo;
      fc.template br_pair<q>(bq, bo);
      S::st2(po + int(q * N), fma(so, fv(qq), bq), fma(sod, hv(qq), fma(h3, cv, h0)));
      S::st2(po + int(o * N), fma(so, fv(oo), bo), fma(sod, hv(oo), fma(-h3, cv, h0)));
    });
    const Real he0 = (sC - hsum) / wq<Real>(0);
    const auto q0 = std::integral_constant<int, 0>{};
    S::st2(po, fma(so, fv(q0), fc.template br<0>()), fma(sod, hv(q0), sc * (itd * he0 - R.y)));
    reinterpret_cast<__half2 *>(a.rf_out)[n] = r2;
  } else if constexpr (S::kShift) {
    // per unit weight, (f~_q - w_q)/w_q = omt e_q + b_q; stored as the
    // remainder scale ((f~_q - w_q)/w_q - drho)
    fc.fold(Real(S::kScale), drho);
    const Real so = Real(S::kScale) * fc.omt;
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      S::template st_raw<q>(fo + int(q * N), fma(so, fv(qc), fc.template br<q>()));
    });
  } else {
    fc.fold(Real(1), Real(0));
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      S::template st_f<q>(fo + int(q * N), fc.template post<q>(fv(qc)));
    });
  }
  if constexpr (S::kShift && !SOLUTE) a.rf_out[n] = float(drho);

  if constexpr (SOLUTE && !S::kShift) {
    T *__restrict__ ho = static_cast<T *>(a.h_out) + n;
    const Real vs0 = fc.Vp[0] + gx, vs1 = fc.Vp[1] + gy, vs2 = fc.Vp[2] + gz;
    const Real itd = a.inv_tau_D;
    // h^eq of the moving directions; the rest component takes the remainder
    // so that sum_q h^eq_q = sum_q h_q holds to rounding (the weights rounded
    // to the collision type sum to 1 + 1.5e-8 in FP32, which would otherwise
    // create solute at every collision)
    Real hsum = Real(0);
    Unroll<1, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const Real cv = Real(cx(q)) * vs0 + Real(cy(q)) * vs1 + Real(cz(q)) * vs2;
      const Real heq = wq<Real>(q) * sC * (Real(1) + Real(3) * cv);
      hsum += heq;
      const Real h = hv(qc);
      S::template st_h<q>(ho + int(q * N), h + (heq - h) * itd);
    });
    {
      const Real h = hv(std::integral_constant<int, 0>{});
      S::template st_h<0>(ho, h + ((sC - hsum) - h) * itd);
    }
  }
  if (a.fields) write_fields(a.fields, N, n, rho, fc.Vp, C, nu);
  if constexpr (VOUT) {
    vout[0] = V[0];
    vout[1] = V[1];
    vout[2] = V[2];
    vout[3] = fc.Vp[0];
    vout[4] = fc.Vp[1];
    vout[5] = fc.Vp[2];
  }
}

// The rows of a cell's K^-1 for the velocity solve. With a full tensor, with
// the Forchheimer drag, in the kernel that also advances further solute
// species, and with 16-bit paired storage, they are loaded with the cell's
// other static fields, before the moments, so their latency hides behind the
// gather (loaded inside the solve they were a second wait per cell: 256^3
// FP32 0.955 -> 0.862 ms, FP16 0.738 -> 0.675 ms, 128^3 Forchheimer 0.136 ->
// 0.122 ms, three species 0.230 -> 0.221 ms, 128^3 FP16 0.0985 -> 0.0914 ms);
// the three rows of a plain diagonal tensor with FP32/FP64 storage stay in the
// solve, where the register budget prefers them (128^3 FP32 0.1126 ms,
// 0.1165 ms early).
template <class Real, int KMODE, bool SPEC = false, bool PAIRED = false>
struct KinvRows {
  static constexpr bool kEarly =
      KMODE == KM_SPD || KMODE == KM_FORCH || ((SPEC || PAIRED) && KMODE == KM_DIAG);
  Real v[kEarly ? 6 : 1];
  __device__ __forceinline__ void load(const Real *kinv, unsigned N, unsigned n) {
    if constexpr (kEarly)
      for (int r = 0; r < 6; ++r) v[r] = __ldg(kinv + size_t(r) * N + n);
  }
  __device__ __forceinline__ Real row(const Real *kinv, unsigned N, unsigned n, int r) const {
    if constexpr (kEarly)
      return v[r];
    else
      return __ldg(kinv + size_t(r) * N + n);
  }
};

// update_cell for 16-bit storage with solute (the paired layout): one 32-bit
// load brings f_q and h_q of a source cell, one more its reference pair, and
// both lattices are gathered per unit weight, d[q] = (f_q - w_q)/w_q and
// hh[q] = h_q/w_q (remainder + the source's reference).
template <class S, int KMODE, int FEAT>
__device__ __forceinline__ void update_cell_paired(const StepArgs<float> &a, unsigned x, unsigned y,
                                                   unsigned z, unsigned n, uint32_t link,
                                                   float &fin_acc, float &fout_acc, float &drho,
                                                   float &sC, bool &open_face,
                                                   float *vout = nullptr) {
  using Real = float;
  using T2 = typename S::T2;
  const unsigned N = a.N;
  const CellGeo g = cell_geo_xyz(x, y, z, a.nx, a.ny, a.nz);
  const T2 *__restrict__ pb = static_cast<const T2 *>(a.f_in) + n;
  const float *__restrict__ rb = a.rf_in + n;  // a __half2 per cell
  Real d[Q], hh[Q];
  const unsigned s_open = a.s_inlet | a.s_outlet;
  open_face = (g.onface & s_open) != 0;
  bool f_simple = link == 0 && !(g.onface & a.f_wall);
  if constexpr ((FEAT & FEAT_OPEN) != 0) f_simple = f_simple && !(g.onface & (a.f_press | a.f_vel));
  const bool both = f_simple && link == 0 && !(g.onface & (a.s_wall | s_open));
  if (both) {
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const float2 p = S::ld2(pb + (int(q * N) + src_delta<q>(g)));
      const float2 r = ld_ref2(rb + src_delta<q>(g));
      d[q] = p.x + r.x;
      hh[q] = p.y + r.y;
    });
  } else if (((FEAT & FEAT_OPEN) != 0) && (g.onface & (a.f_press | a.f_vel))) {
    const Pops<Real> o = gather_open_faces<S>(a, g, n, link);
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      d[q] = o.v[q] * Real(inv_wq(q));
    });
  } else {
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const bool bb = fluid_class<q>(g, link, a.f_wall) == PULL_BOUNCE;
      d[q] = S::ld2(pb + (bb ? int(opp(q) * N) : int(q * N) + src_delta<q>(g))).x +
             ld_ref2(rb + (bb ? 0 : src_delta<q>(g))).x;
    });
  }
  const Real eps = __ldg(a.eps + n);
  const Real gx = __ldg(a.geps + n), gy = __ldg(a.geps + N + n),
             gz = __ldg(a.geps + 2 * size_t(N) + n);
  KinvRows<Real, KMODE, (FEAT & FEAT_SPEC) != 0, true> kr;
  kr.load(a.kinv, N, n);
  Real V[3];
  fluid_moments<true>([&](auto qc) { return d[decltype(qc)::value]; }, drho, V);
  const Real rho = Real(1) + drho;
  const Real ie = rcp(eps);
  if (!both) {
    // the solute classes, per unit weight; the fluxes carry the weights
    const Real vi0 = V[0] + gx, vi1 = V[1] + gy, vi2 = V[2] + gz;
    const Real own = ld_ref2(rb).y;
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const int cls = solute_class<q>(g, link, a.s_wall, a.s_inlet, a.s_outlet);
      Real v;
      if (cls == PULL_CELL) {
        v = S::ld2(pb + (int(q * N) + src_delta<q>(g))).y + ld_ref2(rb + src_delta<q>(g)).y;
      } else if (cls == PULL_BOUNCE) {
        v = S::ld2(pb + int(opp(q) * N)).y + own;
      } else if (cls == PULL_INLET) {
        // entering through an inlet face: h^eq at C_in with the cell's bare
        // streamed velocity plus D grad(eps)/eps
        const Real cv = Real(cx(q)) * vi0 + Real(cy(q)) * vi1 + Real(cz(q)) * vi2;
        v = eps * a.C_in * (Real(1) + Real(3) * cv);
        fin_acc += wq<Real>(q) * (v - (S::ld2(pb + int(opp(q) * N)).y + own));
      } else {
        // outlet: the cell's own post-collision value (zero gradient)
        v = S::ld2(pb + int(q * N)).y + own;
        fout_acc += wq<Real>(q) * ((S::ld2(pb + int(opp(q) * N)).y + own) - v);
      }
      hh[q] = v;
    });
  }
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    sC = fma(wq<Real>(q), hh[q], sC);
  });
  collide_tail<S, KMODE, true, (FEAT & FEAT_SPEC) != 0>(
      a, n, g, [&](auto qc) { return d[decltype(qc)::value]; },
      [&](auto qc) { return hh[decltype(qc)::value]; },
      [&](int r) { return kr.row(a.kinv, N, n, r); }, drho, rho, V, ie, eps, sC, gx, gy, gz,
      vout);
}

// The per-cell update of one step from global memory: stream f (and h),
// moments, viscosity, colour gradient, V' and the Darcy force, fluid and
// solute collision, store; accumulates the cell's flux and totals.
template <class S, int KMODE, bool SOLUTE, int FEAT = 0>
__device__ __forceinline__ void update_cell_sep(const StepArgs<typename S::Real> &a, unsigned x,
                                            unsigned y, unsigned z, unsigned n, uint32_t link,
                                            typename S::Real &fin_acc,
                                            typename S::Real &fout_acc, typename S::Real &drho,
                                            typename S::Real &sC, bool &open_face,
                                            typename S::Real *vout = nullptr) {
  using Real = typename S::Real;
  using T = typename S::T;
  const unsigned N = a.N;
  const CellGeo g = cell_geo_xyz(x, y, z, a.nx, a.ny, a.nz);
  const T *__restrict__ fb = static_cast<const T *>(a.f_in) + n;
  Real d[Q];
  // FEAT_OPEN: the lattice has pressure or velocity faces. A separate
  // instantiation keeps the code of the lattices without them as it is (any
  // extra branch in this gather changes the register allocation of the
  // plain path at its 80-register cap and costs it ~15 %).
  // 16-bit storage: d[q] = (f_q - w_q)/w_q = g_q + the source cell's reference
  auto gather_cells = [&]() {
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      if constexpr (S::kShift)
        d[q] = S::template ld_e<q>(fb + (int(q * N) + src_delta<q>(g))) +
               __ldg(a.rf_in + (long long)n + src_delta<q>(g));
      else
        d[q] = S::template ld_f<q>(fb + (int(q * N) + src_delta<q>(g)));
    });
  };
  auto gather_bounce = [&]() {
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const bool bb = fluid_class<q>(g, link, a.f_wall) == PULL_BOUNCE;
      if constexpr (S::kShift)
        d[q] = S::template ld_e<q>(fb + (bb ? int(opp(q) * N) : int(q * N) + src_delta<q>(g))) +
               __ldg(a.rf_in + (long long)n + (bb ? 0 : src_delta<q>(g)));
      else
        d[q] = S::template ld_f<q>(fb + (bb ? int(opp(q) * N) : int(q * N) + src_delta<q>(g)));
    });
  };
  if constexpr (!(FEAT & FEAT_OPEN)) {
    // every source is a cell, or bounce-back
    if (link == 0 && !(g.onface & a.f_wall))
      gather_cells();
    else
      gather_bounce();
  } else {
    if (link == 0 && !(g.onface & (a.f_wall | a.f_press | a.f_vel))) {
      gather_cells();
    } else if (g.onface & (a.f_press | a.f_vel)) {
      const Pops<Real> o = gather_open_faces<S>(a, g, n, link);
      Unroll<0, Q>::run([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        d[q] = S::kShift ? o.v[q] * Real(inv_wq(q)) : o.v[q];
      });
    } else {
      gather_bounce();
    }
  }
  // every load of the interior path is issued before any arithmetic, so a
  // warp keeps its 38 population rows and static fields in flight together
  const Real eps = __ldg(a.eps + n);
  KinvRows<Real, KMODE, (FEAT & FEAT_SPEC) != 0> kr;
  kr.load(a.kinv, N, n);
  Real hh[SOLUTE ? Q : 1];
  Real gx = Real(0), gy = Real(0), gz = Real(0);
  const T *__restrict__ hb = static_cast<const T *>(a.h_in) + n;
  const unsigned s_open = a.s_inlet | a.s_outlet;
  const bool h_simple = SOLUTE && link == 0 && !(g.onface & (a.s_wall | s_open));
  if (SOLUTE) {
    gx = __ldg(a.geps + n);
    gy = __ldg(a.geps + N + n);
    gz = __ldg(a.geps + 2 * size_t(N) + n);
    open_face = (g.onface & s_open) != 0;
    if (h_simple) {
      Unroll<0, Q>::run([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        hh[SOLUTE ? q : 0] = S::template ld_h<q>(hb + (int(q * N) + src_delta<q>(g)));
      });
    }
  }
  Real V[3];
  fluid_moments<S::kShift>([&](auto qc) { return d[decltype(qc)::value]; }, drho, V);
  const Real rho = Real(1) + drho;
  const Real ie = rcp(eps);

  if constexpr (SOLUTE) {
    if (!h_simple) {
      const Real vi0 = V[0] + gx, vi1 = V[1] + gy, vi2 = V[2] + gz;
      Unroll<0, Q>::run([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const int cls = solute_class<q>(g, link, a.s_wall, a.s_inlet, a.s_outlet);
        Real v;
        if (cls == PULL_CELL) {
          v = S::template ld_h<q>(hb + (int(q * N) + src_delta<q>(g)));
        } else if (cls == PULL_BOUNCE) {
          v = S::template ld_h<opp(q)>(hb + int(opp(q) * N));
        } else if (cls == PULL_INLET) {
          // entering through an inlet face: h^eq at C_in with the cell's
          // bare streamed velocity plus D grad(eps)/eps
          const Real cv = Real(cx(q)) * vi0 + Real(cy(q)) * vi1 + Real(cz(q)) * vi2;
          v = wq<Real>(q) * eps * a.C_in * (Real(1) + Real(3) * cv);
          fin_acc += v - S::template ld_h<opp(q)>(hb + int(opp(q) * N));
        } else {
          // outlet: the cell's own post-collision value (zero gradient)
          v = S::template ld_h<q>(hb + int(q * N));
          fout_acc += S::template ld_h<opp(q)>(hb + int(opp(q) * N)) - v;
        }
        hh[SOLUTE ? q : 0] = v;
      });
    }
    Unroll<0, Q>::run([&](auto qc) { sC += hh[SOLUTE ? decltype(qc)::value : 0]; });
  }
  collide_tail<S, KMODE, SOLUTE, (FEAT & FEAT_SPEC) != 0>(
      a, n, g, [&](auto qc) { return d[decltype(qc)::value]; },
      [&](auto qc) { return hh[SOLUTE ? decltype(qc)::value : 0]; },
      [&](int r) { return kr.row(a.kinv, N, n, r); }, drho, rho, V, ie, eps, sC, gx, gy, gz,
      vout);
}

template <class S, int KMODE, bool SOLUTE, int FEAT = 0>
__device__ __forceinline__ void update_cell(const StepArgs<typename S::Real> &a, unsigned x,
                                            unsigned y, unsigned z, unsigned n, uint32_t link,
                                            typename S::Real &fin_acc,
                                            typename S::Real &fout_acc, typename S::Real &drho,
                                            typename S::Real &sC, bool &open_face,
                                            typename S::Real *vout = nullptr) {
  if constexpr (S::kShift && SOLUTE)
    update_cell_paired<S, KMODE, FEAT>(a, x, y, z, n, link, fin_acc, fout_acc, drho, sC, open_face,
                                       vout);
  else
    update_cell_sep<S, KMODE, SOLUTE, FEAT>(a, x, y, z, n, link, fin_acc, fout_acc, drho, sC,
                                            open_face, vout);
}

// Solute species sp >= 1 of one cell, after the fluid and species 0 of the
// same step (Eqs. equild, boltzeqD for each species, reading R24): each
// species is its own D3Q19 lattice with its own tau_D and inlet
// concentration; all share the cell's V' (vel[3..5]) and, for populations
// entering through an inlet face, its bare streamed velocity V (vel[0..2]).
// The gather with its boundary classes, C = sum_q h_q / eps, h^eq at V* = V' +
// D_s grad(eps)/eps with the rest component as the remainder, BGK.
template <class S>
__device__ __forceinline__ void species_update(const StepArgs<typename S::Real> &a, int sp,
                                               unsigned x, unsigned y, unsigned z, unsigned n,
                                               uint32_t link, const typename S::Real (&vel)[6],
                                               typename S::Real &fin_acc,
                                               typename S::Real &fout_acc, typename S::Real &sC,
                                               bool &open_face) {
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
    const Real vi0 = vel[0] + gx, vi1 = vel[1] + gy, vi2 = vel[2] + gz;
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
  const Real vs0 = vel[3] + gx, vs1 = vel[4] + gy, vs2 = vel[5] + gz;
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

// One time step for every non-solid cell (see update_cell).
// Launch: block (BX, BY) of STEP_BLOCK threads with BX a multiple of 32,
// grid (ceil(nx/BX), ceil(ny/BY), nz); a warp covers 32 consecutive x of one
// row. Six resident 128-thread blocks per SM (at most 85 registers a
// thread): measured on GB300 at 128^3 this is 1.1x faster than the
// unconstrained build (112 registers), since the kernel is bound by loads in
// flight, and a little faster than 256-thread blocks at the same occupancy.
template <class S, int KMODE, bool SOLUTE, int FEAT>
__global__ void __launch_bounds__(STEP_BLOCK, 6) step_kernel(const StepArgs<typename S::Real> a) {
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
  Real fin_acc = Real(0), fout_acc = Real(0), drho = Real(0), sC = Real(0);
  bool open_face = false;
  Real vel[6];
  if (live)
    update_cell<S, KMODE, SOLUTE, FEAT>(a, x, y, z, n, link, fin_acc, fout_acc, drho, sC,
                                        open_face, (FEAT & FEAT_SPEC) ? vel : nullptr);
  warp_reductions(a, warp_gid, open_face, fin_acc, fout_acc, drho, sC);
  if constexpr ((FEAT & FEAT_SPEC) != 0) {
    // further species, each with its per-warp flux slots and finite check
    const unsigned lane = threadIdx.x & 31u;
    for (int sp = 1; sp < a.species; ++sp) {
      Real fin_s = Real(0), fout_s = Real(0), sC_s = Real(0);
      bool of = false;
      if (live) species_update<S>(a, sp, x, y, z, n, link, vel, fin_s, fout_s, sC_s, of);
      if (a.flux && __any_sync(0xffffffffu, of)) {
        const Real si = warp_sum(fin_s), so = warp_sum(fout_s);
        if (lane == 0) {
          double *slot = a.flux_slots + size_t(sp) * a.slot_stride + 2 * size_t(warp_gid);
          slot[0] += double(si);
          slot[1] += double(so);
        }
      }
      if (a.reduce) {
        const Real c = warp_sum(sC_s);
        if (lane == 0 && !isfinite(c)) atomicOr(&a.state->status, 1u);
      }
    }
  }
}

// Post-stream density for the colour gradient (flowchart: stream -> moments
// -> gradient): rhohat = sum_q f_q(x - c_q), solid cells = wall_rho.
template <class S>
__global__ void __launch_bounds__(BLOCK) rhohat_kernel(const StepArgs<typename S::Real> a,
                                                       typename S::Real *rhohat) {
  using Real = typename S::Real;
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  if (n >= a.N) return;
  uint32_t link = a.link ? __ldg(a.link + n) : 0u;
  if (link >> 31) {
    rhohat[n] = a.wall_rho;
    return;
  }
  const CellGeo g = cell_geo(n, a.nx, a.ny, a.nz);
  Real d[Q];
  gather_f<S>(static_cast<const typename S::T *>(a.f_in), a.N, n, g, link, a.f_wall, d, a.rf_in,
              a.paired != 0);
  Real s = Real(0);
  Unroll<0, Q>::run([&](auto qc) { s += d[decltype(qc)::value]; });
  rhohat[n] = Real(1) + s;
}

// ------------------------------------------------------------------------
// Initialisation (flowchart step c): f = f^eq, h = h^eq.
// ------------------------------------------------------------------------
template <class Real>
struct InitArgs {
  const float *rho0, *u0, *C0, *f_scale;  // device copies of the caller's arrays
  const uint8_t *type;                      // NULL unless free surface
};

template <class S, int KMODE, bool SOLUTE>
__global__ void __launch_bounds__(BLOCK) init_kernel(const StepArgs<typename S::Real> a,
                                                     const InitArgs<typename S::Real> in) {
  using Real = typename S::Real;
  using T = typename S::T;
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  const unsigned N = a.N;
  if (n >= N) return;
  T *fout = static_cast<T *>(a.f_out);
  T *fout2 = static_cast<T *>(const_cast<void *>(a.f_in));  // both buffers get the same state
  const bool solid = a.link && (__ldg(a.link + n) >> 31);
  const bool empty = in.type && in.type[n] == CELL_EMPTY;
  if constexpr (S::kShift && SOLUTE) {
    // paired layout: (f, h) remainders per direction, FP16 reference pairs
    using T2 = typename S::T2;
    T2 *p1 = static_cast<T2 *>(a.f_out) + n;
    T2 *p0 = static_cast<T2 *>(const_cast<void *>(a.f_in)) + n;
    if (solid || empty) {
      // absolute populations 0: references (-1, 0), remainders 0
      Unroll<0, Q>::run([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        S::st2(p1 + size_t(q) * N, 0.0f, 0.0f);
        S::st2(p0 + size_t(q) * N, 0.0f, 0.0f);
      });
      const __half2 r2 = __floats2half2_rn(-1.0f, 0.0f);
      reinterpret_cast<__half2 *>(a.rf_out)[n] = r2;
      reinterpret_cast<__half2 *>(const_cast<float *>(a.rf_in))[n] = r2;
      if (a.fields) zero_fields(a.fields, N, n);
      return;
    }
  }
  if (solid || empty) {
    // absolute populations 0 (FP16/BF16: reference -1, remainders 0)
    const Real shift = S::kShift ? Real(-1) : Real(0);
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      S::template st_f<q>(fout + size_t(q) * N + n, -wq<Real>(q) - wq<Real>(q) * shift);
      S::template st_f<q>(fout2 + size_t(q) * N + n, -wq<Real>(q) - wq<Real>(q) * shift);
    });
    if constexpr (S::kShift) {
      a.rf_out[n] = -1.0f;
      const_cast<float *>(a.rf_in)[n] = -1.0f;
      if (SOLUTE) {
        a.rh_out[n] = 0.0f;
        const_cast<float *>(a.rh_in)[n] = 0.0f;
      }
    }
    if (SOLUTE) {
      Unroll<0, Q>::run([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        S::template st_h<q>(static_cast<T *>(a.h_out) + size_t(q) * N + n, Real(0));
        S::template st_h<q>(const_cast<T *>(static_cast<const T *>(a.h_in)) + size_t(q) * N + n,
                            Real(0));
      });
    }
    if (a.fields) zero_fields(a.fields, N, n);
    return;
  }
  const CellGeo g = cell_geo(n, a.nx, a.ny, a.nz);
  const Real rho = Real(in.rho0[n]);
  const Real u[3] = {Real(in.u0[3 * size_t(n)]), Real(in.u0[3 * size_t(n) + 1]),
                     Real(in.u0[3 * size_t(n) + 2])};
  const Real eps = a.eps[n];
  const Real C = SOLUTE ? Real(in.C0[n]) : Real(0);
  const Real tau = tau_of(a, C);  // a.t = 0
  FluidCollide<Real> fc;
  fc.F[0] = fc.F[1] = fc.F[2] = Real(0);
  if (a.A != Real(0)) colour_gradient(a.rhohat, n, g, a.f_wall, a.wall_rho, fc.F);
  fc.drho = rho - Real(1);
  fc.rho = rho;
  fc.ie = Real(1) / eps;
  fc.Vp[0] = u[0]; fc.Vp[1] = u[1]; fc.Vp[2] = u[2];
  fc.uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  fc.Fn = sqrt(fc.F[0] * fc.F[0] + fc.F[1] * fc.F[1] + fc.F[2] * fc.F[2]);
  fc.st = (a.A != Real(0)) && fc.Fn > st_threshold<Real>();
  fc.stc = fc.st ? a.A * eps * tau : Real(0);
  fc.iFn = fc.st ? Real(1) / fc.Fn : Real(0);
  Real devs[Q];
  Real dsum = Real(0);
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    Real dev = fc.template feq_dev<q>();
    if (in.f_scale) {
      const Real sc = Real(in.f_scale[size_t(q) * N + n]);
      dev = (dev + wq<Real>(q)) * sc - wq<Real>(q);
    }
    devs[q] = dev;
    dsum += dev;
  });
  if constexpr (S::kShift && SOLUTE) {
    const Real vs0 = u[0] + a.geps[n], vs1 = u[1] + a.geps[N + n], vs2 = u[2] + a.geps[2 * size_t(N) + n];
    Real hs[Q];
    Real hsum = Real(0);
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const Real cv = Real(cx(q)) * vs0 + Real(cy(q)) * vs1 + Real(cz(q)) * vs2;
      hs[q] = wq<Real>(q) * eps * C * (Real(1) + Real(3) * cv);
      hsum += hs[q];
    });
    // remainders per unit weight against the FP16-rounded references
    const __half2 r2 = __floats2half2_rn(dsum, hsum);
    const float2 R = __half22float2(r2);
    using T2 = typename S::T2;
    T2 *p1 = static_cast<T2 *>(a.f_out) + n;
    T2 *p0 = static_cast<T2 *>(const_cast<void *>(a.f_in)) + n;
    const Real sc = Real(S::kScale);
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const Real gf = sc * (devs[q] * Real(inv_wq(q)) - R.x);
      const Real gh = sc * (hs[q] * Real(inv_wq(q)) - R.y);
      S::st2(p1 + size_t(q) * N, gf, gh);
      S::st2(p0 + size_t(q) * N, gf, gh);
    });
    reinterpret_cast<__half2 *>(a.rf_out)[n] = r2;
    reinterpret_cast<__half2 *>(const_cast<float *>(a.rf_in))[n] = r2;
    if (a.fields) write_fields(a.fields, N, n, rho, u, C, (tau - Real(0.5)) / Real(3));
    return;
  }
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const Real v = devs[q] - (S::kShift ? wq<Real>(q) * dsum : Real(0));
    S::template st_f<q>(fout + size_t(q) * N + n, v);
    S::template st_f<q>(fout2 + size_t(q) * N + n, v);
  });
  if constexpr (S::kShift) {
    a.rf_out[n] = float(dsum);
    const_cast<float *>(a.rf_in)[n] = float(dsum);
  }
  if (SOLUTE) {
    const Real vs0 = u[0] + a.geps[n], vs1 = u[1] + a.geps[N + n], vs2 = u[2] + a.geps[2 * size_t(N) + n];
    Real hs[Q];
    Real hsum = Real(0);
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const Real cv = Real(cx(q)) * vs0 + Real(cy(q)) * vs1 + Real(cz(q)) * vs2;
      hs[q] = wq<Real>(q) * eps * C * (Real(1) + Real(3) * cv);
      hsum += hs[q];
    });
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const Real h = hs[q] - (S::kShift ? wq<Real>(q) * hsum : Real(0));
      S::template st_h<q>(static_cast<T *>(a.h_out) + size_t(q) * N + n, h);
      S::template st_h<q>(const_cast<T *>(static_cast<const T *>(a.h_in)) + size_t(q) * N + n, h);
    });
    if constexpr (S::kShift) {
      a.rh_out[n] = float(hsum);
      const_cast<float *>(a.rh_in)[n] = float(hsum);
    }
  }
  if (a.fields) write_fields(a.fields, N, n, rho, u, C, (tau - Real(0.5)) / Real(3));
}

// ------------------------------------------------------------------------
// Populations <-> absolute FP64, totals and the neighbour export.
// ------------------------------------------------------------------------
// The reference of cell n in a view (0 without references).
__device__ __forceinline__ double pop_ref(const PopView &v, unsigned n) {
  if (!v.ref) return 0.0;
  if (v.ref_pair) {
    const __half2 r = static_cast<const __half2 *>(v.ref)[n];
    return double(v.off ? __high2float(r) : __low2float(r));
  }
  return double(static_cast<const float *>(v.ref)[n]);
}
template <class S>
__device__ __forceinline__ typename S::T pop_at(const PopView &v, size_t i) {
  return static_cast<const typename S::T *>(v.p)[size_t(v.stride) * i + v.off];
}

template <class S>
__global__ void to_f64_kernel(const PopView v, double *dst, unsigned N, int lattice) {
  const size_t i = size_t(blockIdx.x) * BLOCK + threadIdx.x;
  if (i >= size_t(Q) * N) return;
  const int q = int(i / N);
  const double r = pop_ref(v, unsigned(i % N));
  dst[i] = lattice == 0 ? S::to_f(pop_at<S>(v, i), q, r) : S::to_h(pop_at<S>(v, i), q, r);
}

// per cell: the reference of given FP64 populations (sum of f_q - w_q, or of
// h_q), stored rounded to the view's reference type
static __global__ void ref_from_f64_kernel(const double *src, unsigned N, int lattice,
                                           const PopView v) {
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  if (n >= N) return;
  double s = 0.0;
  for (int q = 0; q < Q; ++q) s += src[size_t(q) * N + n] - (lattice == 0 ? wq<double>(q) : 0.0);
  if (v.ref_pair)
    static_cast<__half *>(const_cast<void *>(v.ref))[2 * size_t(n) + v.off] = __float2half_rn(float(s));
  else
    static_cast<float *>(const_cast<void *>(v.ref))[n] = float(s);
}

template <class S>
__global__ void from_f64_kernel(const double *src, const PopView v, unsigned N, int lattice) {
  const size_t i = size_t(blockIdx.x) * BLOCK + threadIdx.x;
  if (i >= size_t(Q) * N) return;
  const int q = int(i / N);
  const double r = pop_ref(v, unsigned(i % N));
  static_cast<typename S::T *>(const_cast<void *>(v.p))[size_t(v.stride) * i + v.off] =
      lattice == 0 ? S::from_f(src[i], q, r) : S::from_h(src[i], q, r);
}

// Per-block FP64 sums of the fluid mass and the solute over non-solid cells,
// each block taking cells blockIdx.x*BLOCK + tid + k*gridDim.x*BLOCK. A
// cell's 19 stored values are summed in the collision type as deviations
// (FP32 / FP64 storage: f_q - w_q, h_q; 16-bit: the remainders times w_q),
// then mass = 1 + reference + sum, solute = reference + sum in FP64; the
// cell sums, the block's shuffle tree and the finish are FP64.
template <class S>
__global__ void __launch_bounds__(BLOCK) totals_kernel(const PopView f, const PopView h,
                                                       const uint32_t *link, unsigned N,
                                                       double *partials) {
  using Real = typename S::Real;
  __shared__ double sh[BLOCK / 32][2];
  double m = 0.0, s = 0.0;
  for (unsigned n = blockIdx.x * BLOCK + threadIdx.x; n < N; n += gridDim.x * BLOCK) {
    if (link && (link[n] >> 31)) continue;
    Real a = Real(0);
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      a += S::template cv_f<q>(pop_at<S>(f, size_t(q) * N + n));
    });
    m += 1.0 + pop_ref(f, n) + double(a);
    if (h.p) {
      Real b = Real(0);
      Unroll<0, Q>::run([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        b += S::template cv_h<q>(pop_at<S>(h, size_t(q) * N + n));
      });
      s += pop_ref(h, n) + double(b);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_down_sync(0xffffffffu, m, o);
    s += __shfl_down_sync(0xffffffffu, s, o);
  }
  const unsigned w = threadIdx.x >> 5;
  if ((threadIdx.x & 31u) == 0) {
    sh[w][0] = m;
    sh[w][1] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tm = 0.0, ts = 0.0;
    for (unsigned k = 0; k < BLOCK / 32; ++k) {
      tm += sh[k][0];
      ts += sh[k][1];
    }
    partials[2 * size_t(blockIdx.x)] = tm;
    partials[2 * size_t(blockIdx.x) + 1] = ts;
  }
}

// Fixed-order sum of nblk x K partials by one block of FINISH_THREADS
// threads (thread t sums partials t, t + FINISH_THREADS, ..., then a fixed
// tree), so the result does not depend on timing.
constexpr int FINISH_THREADS = 1024;
template <int K>
__global__ void __launch_bounds__(FINISH_THREADS) finish_sum_kernel(const double *partials,
                                                                    unsigned nblk, double *out) {
  __shared__ double sh[FINISH_THREADS][K];
  double acc[K];
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (unsigned b = threadIdx.x; b < nblk; b += FINISH_THREADS)
    for (int k = 0; k < K; ++k) acc[k] += partials[size_t(b) * K + k];
  for (int k = 0; k < K; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int s = FINISH_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < K; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
    __syncthreads();
  }
  if (threadIdx.x < K) out[threadIdx.x] = sh[0][threadIdx.x];
}

template <class Real>
__global__ void neighbors_kernel(const StepArgs<Real> a, int lattice, int32_t *src) {
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  const unsigned N = a.N;
  if (n >= N) return;
  const uint32_t link = a.link ? a.link[n] : 0u;
  const CellGeo g = cell_geo(n, a.nx, a.ny, a.nz);
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    int32_t v;
    if (link >> 31) {
      v = -1;
    } else {
      const int cls = lattice == 0 ? fluid_class_open<q>(g, link, a.f_wall, a.f_vel, a.f_press)
                                   : solute_class<q>(g, link, a.s_wall, a.s_inlet, a.s_outlet);
      v = cls == PULL_CELL ? int32_t((long long)n + src_delta<q>(g)) : -(1 + cls);
    }
    src[size_t(q) * N + n] = v;
  });
}

}  // namespace lbgb
