// Shared device-side definitions of the GB300 lattice-Boltzmann library:
// the D3Q19 velocity set, population storage formats and kernel arguments.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbgb {

constexpr int Q = 19;
constexpr int BLOCK = 256;       // threads per block of the per-cell helper kernels
constexpr int STEP_BLOCK = 128;  // threads per block of the step kernels

// D3Q19 velocity set in the paper's (orientation i, reference plane p) order
// (Section 2.1, Fig. d3q19): q = 0 rest; q = 1 + 6p + (i-1) with planes
// p = 0 (x-y), 1 (y-z), 2 (z-x); i = 1..4 the plane's diagonals
// counter-clockwise starting at (+first, +second) axis; i = 5, 6 = +/- the
// plane's first axis. The figure is not reproduced in the paper's text, so
// this ordering is a reading; the physics does not depend on it.
__host__ __device__ constexpr int cx(int q) {
  constexpr int t[Q] = {0, 1, -1, -1, 1, 1, -1, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0};
  return t[q];
}
__host__ __device__ constexpr int cy(int q) {
  constexpr int t[Q] = {0, 1, 1, -1, -1, 0, 0, 1, -1, -1, 1, 1, -1, 0, 0, 0, 0, 0, 0};
  return t[q];
}
__host__ __device__ constexpr int cz(int q) {
  constexpr int t[Q] = {0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 1, -1, -1, 1, 1, -1};
  return t[q];
}
// opposite direction: diagonals i <-> i+2 (mod 4), axis 5 <-> 6, same plane
__host__ __device__ constexpr int opp(int q) {
  constexpr int t[Q] = {0, 3, 4, 1, 2, 6, 5, 9, 10, 7, 8, 12, 11, 15, 16, 13, 14, 18, 17};
  return t[q];
}
// weights after Eq. equilc2: 1/3 rest, 1/18 axis, 1/36 diagonal
template <class R>
__host__ __device__ constexpr R wq(int q) {
  return q == 0 ? R(1) / R(3)
                : ((cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q)) == 1 ? R(1) / R(18)
                                                                        : R(1) / R(36));
}
// 1/w_q, exact small integers
__host__ __device__ constexpr int inv_wq(int q) {
  return q == 0 ? 3 : ((cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q)) == 1 ? 18 : 36);
}

// Faces of the box, bit index: 0 x-low, 1 x-high, 2 y-low, 3 y-high, 4 z-low, 5 z-high.
// faces_crossed(q): faces a pull along c_q may leave through (the source is
// x - c_q, so c = +1 looks at the low face and c = -1 at the high face).
__host__ __device__ constexpr unsigned faces_crossed(int q) {
  return (cx(q) > 0 ? 1u : 0u) | (cx(q) < 0 ? 2u : 0u) | (cy(q) > 0 ? 4u : 0u) |
         (cy(q) < 0 ? 8u : 0u) | (cz(q) > 0 ? 16u : 0u) | (cz(q) < 0 ? 32u : 0u);
}
// faces the step x + c_q may leave through (stencils that look forward)
__host__ __device__ constexpr unsigned faces_ahead(int q) { return faces_crossed(opp(q)); }

// ------------------------------------------------------------------------
// Population storage formats. ld_f returns f_q - w_q, ld_h returns h_q, both
// in the collision type Real; st_* take the same quantities.
// ------------------------------------------------------------------------
// FP32 / FP64 populations are stored with plain stores: measured on GB300 at
// 128^3 they step 1.3 % faster than with the evict-first hint (the written
// lines stay in L2 and drain behind the next loads).
struct StoreF32 {
  using T = float;
  using Real = float;
  static constexpr int id = 0;
  static constexpr bool kShift = false;
  static constexpr float kScale = 1.0f;
  template <int q> __device__ __forceinline__ static Real cv_f(T v) { return v; }
  template <int q> __device__ __forceinline__ static Real cv_h(T v) { return v; }
  template <int q> __device__ __forceinline__ static Real ld_f(const T *p) { return __ldg(p); }
  template <int q> __device__ __forceinline__ static void st_f(T *p, Real v) { *p = v; }
  template <int q> __device__ __forceinline__ static Real ld_h(const T *p) { return __ldg(p); }
  template <int q> __device__ __forceinline__ static void st_h(T *p, Real v) { *p = v; }
  __host__ __device__ static double to_f(T v, int q, double = 0.0) { return double(v) + wq<double>(q); }
  __host__ __device__ static T from_f(double f, int q, double = 0.0) { return T(f - wq<double>(q)); }
  __host__ __device__ static double to_h(T v, int, double = 0.0) { return double(v); }
  __host__ __device__ static T from_h(double h, int, double = 0.0) { return T(h); }
};

struct StoreF64 {
  using T = double;
  using Real = double;
  static constexpr int id = 1;
  static constexpr bool kShift = false;
  static constexpr float kScale = 1.0f;
  template <int q> __device__ __forceinline__ static Real cv_f(T v) { return v; }
  template <int q> __device__ __forceinline__ static Real cv_h(T v) { return v; }
  template <int q> __device__ __forceinline__ static Real ld_f(const T *p) { return __ldg(p); }
  template <int q> __device__ __forceinline__ static void st_f(T *p, Real v) { *p = v; }
  template <int q> __device__ __forceinline__ static Real ld_h(const T *p) { return __ldg(p); }
  template <int q> __device__ __forceinline__ static void st_h(T *p, Real v) { *p = v; }
  __host__ __device__ static double to_f(T v, int q, double = 0.0) { return v + wq<double>(q); }
  __host__ __device__ static T from_f(double f, int q, double = 0.0) { return f - wq<double>(q); }
  __host__ __device__ static double to_h(T v, int, double = 0.0) { return v; }
  __host__ __device__ static T from_h(double h, int, double = 0.0) { return h; }
};

// FP16 / BF16: each cell also keeps a reference per lattice (its density
// deviation rho - 1 for f, its solute content sum_q h_q for h), and the
// 16-bit populations hold the remainder g_q = (f_q - w_q)/w_q - ref (resp.
// h_q/w_q - ref): the conserved parts never pass through the short mantissa.
// ld_*/st_* below convert w_q g_q (rows with FP32 references: lattices without
// solute, species 1 ..); ld_e / st_raw the remainder itself, ld2 / st2 the
// (f, h) pairs of the paired layout with its FP16 reference pairs.
struct StoreF16 {
  using T = __half;
  using Real = float;
  static constexpr int id = 2;
  static constexpr bool kShift = true;
  // remainders are stored times 2^12 (exact), which keeps the small ones of
  // slow regions out of FP16's subnormal range; |g| up to 16 fits
  static constexpr float kScale = 4096.0f;
  template <int q> __device__ __forceinline__ static Real cv_f(T v) {
    return __half2float(v) * (wq<float>(q) / kScale);
  }
  template <int q> __device__ __forceinline__ static Real cv_h(T v) {
    return __half2float(v) * (wq<float>(q) / kScale);
  }
  template <int q> __device__ __forceinline__ static Real ld_f(const T *p) {
    return __half2float(__ldg(p)) * (wq<float>(q) / kScale);
  }
  template <int q> __device__ __forceinline__ static void st_f(T *p, Real v) {
    __stcs(p, __float2half_rn(v * (float(inv_wq(q)) * kScale)));
  }
  template <int q> __device__ __forceinline__ static Real ld_h(const T *p) {
    return __half2float(__ldg(p)) * (wq<float>(q) / kScale);
  }
  template <int q> __device__ __forceinline__ static void st_h(T *p, Real v) {
    __stcs(p, __float2half_rn(v * (float(inv_wq(q)) * kScale)));
  }
  // the remainder g itself (unscaled), and a store of a value already in
  // storage units
  template <int q> __device__ __forceinline__ static Real ld_e(const T *p) {
    return __half2float(__ldg(p)) * (1.0f / kScale);
  }
  template <int q> __device__ __forceinline__ static void st_raw(T *p, Real v) {
    __stcs(p, __float2half_rn(v));
  }
  // the (f, h) pair of the paired layout as unscaled remainders, and a store
  // of a pair already in storage units
  using T2 = __half2;
  __device__ __forceinline__ static float2 ld2(const T2 *p) {
    const float2 v = __half22float2(__ldg(p));
    return make_float2(v.x * (1.0f / kScale), v.y * (1.0f / kScale));
  }
  __device__ __forceinline__ static void st2(T2 *p, float lo, float hi) {
    __stcs(p, __floats2half2_rn(lo, hi));
  }
  // with ref: f = w (g + ref) + w, h = w (g + ref)
  __device__ static double to_f(T v, int q, double ref) { return (double(__half2float(v)) / kScale + ref) * wq<double>(q) + wq<double>(q); }
  __device__ static T from_f(double f, int q, double ref) { return __float2half_rn(float(((f - wq<double>(q)) * inv_wq(q) - ref) * kScale)); }
  __device__ static double to_h(T v, int q, double ref) { return (double(__half2float(v)) / kScale + ref) * wq<double>(q); }
  __device__ static T from_h(double h, int q, double ref) { return __float2half_rn(float((h * inv_wq(q) - ref) * kScale)); }
};

struct StoreBF16 {
  using T = __nv_bfloat16;
  using Real = float;
  static constexpr int id = 3;
  static constexpr bool kShift = true;
  static constexpr float kScale = 1.0f;
  template <int q> __device__ __forceinline__ static Real cv_f(T v) {
    return __bfloat162float(v) * wq<float>(q);
  }
  template <int q> __device__ __forceinline__ static Real cv_h(T v) {
    return __bfloat162float(v) * wq<float>(q);
  }
  template <int q> __device__ __forceinline__ static Real ld_f(const T *p) {
    return __bfloat162float(__ldg(p)) * wq<float>(q);
  }
  template <int q> __device__ __forceinline__ static void st_f(T *p, Real v) {
    __stcs(p, __float2bfloat16_rn(v * float(inv_wq(q))));
  }
  template <int q> __device__ __forceinline__ static Real ld_h(const T *p) {
    return __bfloat162float(__ldg(p)) * wq<float>(q);
  }
  template <int q> __device__ __forceinline__ static void st_h(T *p, Real v) {
    __stcs(p, __float2bfloat16_rn(v * float(inv_wq(q))));
  }
  template <int q> __device__ __forceinline__ static Real ld_e(const T *p) {
    return __bfloat162float(__ldg(p));
  }
  template <int q> __device__ __forceinline__ static void st_raw(T *p, Real v) {
    __stcs(p, __float2bfloat16_rn(v));
  }
  using T2 = __nv_bfloat162;
  __device__ __forceinline__ static float2 ld2(const T2 *p) {
    return __bfloat1622float2(__ldg(p));
  }
  __device__ __forceinline__ static void st2(T2 *p, float lo, float hi) {
    __stcs(p, __floats2bfloat162_rn(lo, hi));
  }
  __device__ static double to_f(T v, int q, double ref) { return (double(__bfloat162float(v)) + ref) * wq<double>(q) + wq<double>(q); }
  __device__ static T from_f(double f, int q, double ref) { return __float2bfloat16_rn(float((f - wq<double>(q)) * inv_wq(q) - ref)); }
  __device__ static double to_h(T v, int q, double ref) { return (double(__bfloat162float(v)) + ref) * wq<double>(q); }
  __device__ static T from_h(double h, int q, double ref) { return __float2bfloat16_rn(float(h * inv_wq(q) - ref)); }
};

// The FP16 reference pair (f, h) of a cell in the paired layout; the
// references are FP16 for both 16-bit formats (the remainders are formed
// against the rounded values, so their precision only sets how small the
// remainders are).
__device__ __forceinline__ float2 ld_ref2(const float *p) {
  return __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
}

// ------------------------------------------------------------------------
// Kernel arguments (passed by value).
// ------------------------------------------------------------------------
// permeability modes: no medium, diagonal K^-1, full SPD K^-1, diagonal K^-1
// with Forchheimer drag
enum : int { KM_NONE = 0, KM_DIAG = 1, KM_SPD = 2, KM_FORCH = 3 };
enum : uint8_t { CELL_LIQUID = 0, CELL_INTERFACE = 1, CELL_EMPTY = 2 };

// Device-resident per-context status word.
struct DevState {
  unsigned status;  // bit 0: a checked step met a non-finite mass or solute sum;
                    // bit 1: a bounded wait of the row-pipelined kernel gave up
  unsigned pad;
};

template <class Real>
struct StepArgs {
  int nx, ny, nz;
  unsigned N;
  // face-kind masks over the 6 faces (bit layout of faces_crossed)
  unsigned f_wall;                   // fluid wall faces
  unsigned f_press, f_vel;           // fluid pressure / velocity faces (others periodic)
  unsigned s_wall, s_inlet, s_outlet;  // solute faces
  const void *f_in;
  void *f_out;
  const void *h_in;
  void *h_out;
  const float *rf_in, *rh_in;  // FP16/BF16: per-cell references of the input populations
  float *rf_out, *rh_out;      // ... and of the output populations
  // paired (FP16/BF16 with solute): f_in/f_out hold (f_q, h_q) of species 0
  // as one 32-bit pair per direction and cell, rf_in/rf_out the FP16 pair of
  // references (f, h) per cell (__half2), h_in/h_out species 1 .. only
  // (species s at (s - 1) Q N) with their FP32 references at rh + s N
  int paired;
  const Real *eps;       // N
  const Real *kinv;      // KM_DIAG: 3 x N (xx, yy, zz); KM_SPD: 6 x N (xx, yy, zz, xy, yz, zx)
  const Real *geps;      // 3 x N: D grad(eps)/eps (solute only)
  const uint32_t *link;  // N: bit q = source x - c_q solid; bit 31 = cell solid (NULL: no solids)
  const Real *rhohat;    // N colour-gradient field (A != 0)
  const Real *face;      // per face (2 axis + side): [0, 6) 3 x pressure, [6, 24) velocity xyz,
                         // [24, 30) 3 x pressure minus its rounding to Real
  Real G[3];
  Real tau, tau0, tau1, nu_g, a_h, alpha, beta;
  int visc_law;
  Real A, wall_rho;
  Real forch;           // multiplier of the Ergun coefficient (KM_FORCH)
  Real inv_tau_D, D, C_in;
  long long t;          // step index after the increment
  int reduce;           // form mass / solute totals this step
  int flux;             // inlet/outlet faces present
  float *fields;        // NULL or 6 x N: rho, ux, uy, uz, C, nu
  double *flux_slots;   // 2 per warp of the step launch: cumulative inlet / outlet flux
  DevState *state;
  // Several solute species (kernel feature FEAT_SPEC): spec holds per species
  // [0, 8) 1/tau_D, [8, 16) C_in, [16, 24) D_s / D_0; species s uses the flux
  // slots at flux_slots + s * slot_stride.
  const Real *spec;
  int species;
  unsigned slot_stride;
};

// Free-surface state of one step (Section 3): cell types, liquid mass m,
// liquid fraction lambda and the re-typing scratch.
// Conversion flags: an interface cell that fills or empties, and (re-typing
// pass onwards) an empty cell that has become an interface cell.
enum : uint8_t { FS_NONE = 0, FS_FILL = 1, FS_EMPTYING = 2, FS_NEWCELL = 3 };

template <class Real>
struct FsArgs {
  StepArgs<Real> a;      // fields must be set: rho and V' of every live cell
  uint8_t *type_old;     // read by the step; the last pass settles it to the new type
  uint8_t *type_new;
  Real *m_old;           // read by the step; the last pass settles it to the new mass
  Real *m_new;
  Real *lam;             // lambda(t) in, lambda(t+1) out
  Real *rhohat_w;        // colour-gradient field written by the mass exchange
  uint8_t *flag_a, *flag_b;
  Real *rho_post;        // post-collision density of each live cell (new interface cells:
                         // of their initial populations)
  Real *share;           // excess mass handed to each interface neighbour
  Real *mom;             // rho, V'_x, V'_y, V'_z (4 x N) of each live cell that pulls
                         // from an empty cell, written by the step pass
  unsigned *any;         // nonzero when some cell fills or empties this step
  // Active tiles of FS_TX x FS_TY x FS_TZ cells: the tiles within one tile
  // (26-neighbourhood, wrapped) of a tile holding a liquid or interface cell.
  // The step runs over this step's list; its last pass stamps the tiles of
  // the next step and lists each tile the first time it stamps it.
  const uint32_t *tiles;
  const unsigned *n_tiles;
  uint32_t *next_tiles;
  unsigned *next_n_tiles;
  unsigned *stamp;       // per tile: the step whose list holds it
  unsigned *stamp_ctr;   // steps taken; the next step's stamp is *stamp_ctr + 1 (the
                         // first pass of a step advances it, so a step is launch-invariant)
  unsigned ntx, nty, ntz;
};
constexpr unsigned FS_TX = 32, FS_TY = 1, FS_TZ = 2;
// the tile passes run one block of FS_BLOCK threads per tile (one thread a
// cell), with as many blocks per SM as its 2048 threads and 32 blocks allow
constexpr unsigned FS_BLOCK = FS_TX * FS_TY * FS_TZ;
constexpr unsigned FS_BLOCKS_PER_SM = 2048 / FS_BLOCK < 32 ? 2048 / FS_BLOCK : 32;

}  // namespace lbgb
