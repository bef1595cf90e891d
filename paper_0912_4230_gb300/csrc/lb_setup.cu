// Create-time kernels: validation of the static fields, the inverse
// permeability, the porosity-gradient term of the solute velocity, and the
// per-cell link words (which pull sources are solid).
#include "lb_kernels.cuh"
#include "lb_ops.h"

namespace lbgb {

namespace {

__device__ bool spd3(const double (&M)[3][3]) {
  // Cholesky test
  const double l00s = M[0][0];
  if (!(l00s > 0.0)) return false;
  const double l00 = sqrt(l00s);
  const double l10 = M[1][0] / l00, l20 = M[2][0] / l00;
  const double d1 = M[1][1] - l10 * l10;
  if (!(d1 > 0.0)) return false;
  const double l11 = sqrt(d1);
  const double l21 = (M[2][1] - l20 * l10) / l11;
  const double d2 = M[2][2] - l20 * l20 - l21 * l21;
  return d2 > 0.0;
}

__device__ void load_K(const float *K6, unsigned n, double (&M)[3][3]) {
  const float *k = K6 + 6 * size_t(n);
  M[0][0] = k[0]; M[1][1] = k[1]; M[2][2] = k[2];
  M[0][1] = M[1][0] = k[3];
  M[1][2] = M[2][1] = k[4];
  M[2][0] = M[0][2] = k[5];
}

// the cell x + c_q or -1 when that step leaves through one of the faces in `closed`
__device__ long long step_ahead(const CellGeo &g, unsigned n, int q, unsigned closed) {
  const unsigned ahead = faces_crossed(opp(q));
  if (ahead & g.onface & closed) return -1;
  const int dx = cx(q) > 0 ? g.dxp : (cx(q) < 0 ? g.dxm : 0);
  const int dy = cy(q) > 0 ? g.dyp : (cy(q) < 0 ? g.dym : 0);
  const int dz = cz(q) > 0 ? g.dzp : (cz(q) < 0 ? g.dzm : 0);
  return (long long)n + dx + dy + dz;
}

__global__ void scan_kernel(const SetupArgs a) {
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  if (n >= a.N) return;
  unsigned fl = 0;
  if (a.solid[n]) {
    fl |= 8u;
  } else {
    const float e = a.eps_in[n];
    if (!(e > 0.0f && e <= 1.0f)) fl |= 1u;
    if (a.K6_in) {
      double M[3][3];
      load_K(a.K6_in, n, M);
      if (!spd3(M)) fl |= 2u;
      if (M[0][1] != 0.0 || M[1][2] != 0.0 || M[2][0] != 0.0) fl |= 4u;
    }
  }
  if (fl) atomicOr(a.flags, fl);
}

template <class Real>
__global__ void fields_kernel(const SetupArgs a) {
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  const unsigned N = a.N;
  if (n >= N) return;
  Real *eps = static_cast<Real *>(a.eps);
  const CellGeo g = cell_geo(n, a.nx, a.ny, a.nz);
  const bool solid = a.solid[n] != 0;
  // link word: bit q = the pull source x - c_q (fluid topology) is solid
  uint32_t link = solid ? (1u << 31) : 0u;
  for (int q = 1; q < Q; ++q) {
    const long long s = step_ahead(g, n, opp(q), a.f_wall);
    if (s >= 0 && a.solid[s]) link |= 1u << q;
  }
  a.link[n] = link;
  const double e = solid ? 1.0 : double(a.eps_in[n]);
  eps[n] = Real(e);
  if (a.kinv) {
    Real *ki = static_cast<Real *>(a.kinv);
    double M[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (!solid) load_K(a.K6_in, n, M);
    // inverse of the symmetric matrix by its adjugate
    const double c00 = M[1][1] * M[2][2] - M[1][2] * M[1][2];
    const double c01 = M[0][2] * M[1][2] - M[0][1] * M[2][2];
    const double c02 = M[0][1] * M[1][2] - M[0][2] * M[1][1];
    const double c11 = M[0][0] * M[2][2] - M[0][2] * M[0][2];
    const double c12 = M[0][1] * M[0][2] - M[0][0] * M[1][2];
    const double c22 = M[0][0] * M[1][1] - M[0][1] * M[0][1];
    const double det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
    ki[n] = Real(c00 / det);
    ki[size_t(N) + n] = Real(c11 / det);
    ki[2 * size_t(N) + n] = Real(c22 / det);
    if (a.kmode == KM_SPD) {
      ki[3 * size_t(N) + n] = Real(c01 / det);
      ki[4 * size_t(N) + n] = Real(c12 / det);
      ki[5 * size_t(N) + n] = Real(c02 / det);
    }
  }
  if (a.geps) {
    // D grad(eps)/eps with grad(eps) = 3 sum_q w_q eps(x + c_q) c_q on the
    // solute lattice; solid or out-of-box neighbours contribute eps(x)
    Real *ge = static_cast<Real *>(a.geps);
    double gx = 0, gy = 0, gz = 0;
    if (!solid) {
      for (int q = 1; q < Q; ++q) {
        const long long b = step_ahead(g, n, q, a.s_wall | a.s_open);
        const double eb = (b < 0 || a.solid[b]) ? e : double(a.eps_in[b]);
        const double w3 = 3.0 * wq<double>(q) * eb;
        gx += w3 * cx(q);
        gy += w3 * cy(q);
        gz += w3 * cz(q);
      }
    }
    const double f = a.D / e;
    ge[n] = Real(gx * f);
    ge[size_t(N) + n] = Real(gy * f);
    ge[2 * size_t(N) + n] = Real(gz * f);
  }
}

template <class Real>
__global__ void rhohat_init_k(unsigned N, const uint32_t *link, const float *rho0,
                              const Real *mass, Real wall_rho, Real *rhohat) {
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  if (n >= N) return;
  if (link[n] >> 31)
    rhohat[n] = wall_rho;
  else
    rhohat[n] = mass ? Real(mass[n]) : Real(rho0[n]);
}

unsigned blocks_for(unsigned N) { return (N + BLOCK - 1) / BLOCK; }

}  // namespace

cudaError_t setup_scan(const SetupArgs &a, bool, cudaStream_t s) {
  scan_kernel<<<blocks_for(a.N), BLOCK, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t setup_fields(const SetupArgs &a, bool fp64, cudaStream_t s) {
  if (fp64)
    fields_kernel<double><<<blocks_for(a.N), BLOCK, 0, s>>>(a);
  else
    fields_kernel<float><<<blocks_for(a.N), BLOCK, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t finish_sum(const double *partials, unsigned nblk, int k, double *out, cudaStream_t s) {
  if (k == 2)
    finish_sum_kernel<2><<<1, FINISH_THREADS, 0, s>>>(partials, nblk, out);
  else
    finish_sum_kernel<4><<<1, FINISH_THREADS, 0, s>>>(partials, nblk, out);
  return cudaGetLastError();
}

cudaError_t neighbors(const void *args, bool fp64, int lattice, int32_t *src, unsigned nblk,
                      cudaStream_t s) {
  if (fp64)
    neighbors_kernel<double><<<nblk, BLOCK, 0, s>>>(*static_cast<const StepArgs<double> *>(args),
                                                    lattice, src);
  else
    neighbors_kernel<float><<<nblk, BLOCK, 0, s>>>(*static_cast<const StepArgs<float> *>(args),
                                                   lattice, src);
  return cudaGetLastError();
}

cudaError_t rhohat_init(unsigned N, const uint32_t *link, const float *rho0, const void *mass,
                        double wall_rho, void *rhohat, bool fp64, cudaStream_t s) {
  if (fp64)
    rhohat_init_k<double><<<blocks_for(N), BLOCK, 0, s>>>(
        N, link, rho0, static_cast<const double *>(mass), wall_rho, static_cast<double *>(rhohat));
  else
    rhohat_init_k<float><<<blocks_for(N), BLOCK, 0, s>>>(N, link, rho0,
                                                         static_cast<const float *>(mass),
                                                         float(wall_rho),
                                                         static_cast<float *>(rhohat));
  return cudaGetLastError();
}

}  // namespace lbgb
