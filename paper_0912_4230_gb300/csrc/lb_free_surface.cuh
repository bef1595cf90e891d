// Free-surface kernels (Section 3 of the paper): liquid-mass exchange,
// stream/collide of liquid and interface cells with the reconstruction of
// populations coming from empty cells, and the re-typing of cells whose
// liquid fraction leaves [0, 1]. One step is five passes over the active
// tiles (tiles within one tile of a liquid or interface cell; every cell
// outside them is empty with nothing to do): the mass exchange, the
// stream/collide with the conversion flags, the re-typing, the new interface
// cells and excess mass, and the finish (shares received, liquid fraction,
// the next step's tile list). Each pass needs its neighbours' results of the
// one before; the conversion passes do nothing unless some cell flagged a
// conversion in this step.
#pragma once

#include "lb_kernels.cuh"

namespace lbgb {

// the neighbour x + c_q, or -1 when the step leaves through a wall face or
// lands on a solid cell (bit opp(q) of the link word is the solidity of
// x - c_opp(q) = x + c_q)
template <int q>
__device__ __forceinline__ long long fs_neighbor(const CellGeo &g, unsigned n, uint32_t link,
                                                 unsigned f_wall) {
  if (faces_ahead(q) & g.onface & f_wall) return -1;
  if ((link >> opp(q)) & 1u) return -1;
  return (long long)n + ahead_delta<q>(g);
}

static_assert(FS_BLOCK % 32 == 0 && FS_BLOCK >= 27,
              "whole warps per tile, and a thread for each of the 27 tiles around it");
// With FP32 storage the stream/collide pass keeps 24 warps per SM resident
// (at most 85 registers a thread): on the falling drop 3 % faster than at 96
// registers (20 warps), and no spills. FP64 takes what it needs.
template <class Real>
constexpr unsigned fs_step_blocks() {
  return sizeof(Real) == 4 ? 768 / FS_BLOCK : 1;
}

// Tiles needed by the next step around one cell, as a mask over the 27
// tile offsets (bit (dx+1) + 3(dy+1) + 9(dz+1)): the cell's own tile when
// `self`, and with `halo` also the tiles holding its D3Q19 neighbours (a
// neighbour lies in another tile only when the cell is on that tile face).
__device__ __forceinline__ unsigned fs_tile_mask(unsigned lx, unsigned ly, unsigned lz, bool self,
                                                 bool halo) {
  if (!self && !halo) return 0u;
  unsigned m = 1u << 13;
  if (!halo) return m;
  const int x0 = lx == 0 ? -1 : 0, x1 = lx == FS_TX - 1 ? 1 : 0;
  const int y0 = ly == 0 ? -1 : 0, y1 = ly == FS_TY - 1 ? 1 : 0;
  const int z0 = lz == 0 ? -1 : 0, z1 = lz == FS_TZ - 1 ? 1 : 0;
  for (int dz = z0; dz <= z1; ++dz)
    for (int dy = y0; dy <= y1; ++dy)
      for (int dx = x0; dx <= x1; ++dx)
        if (dx * dx + dy * dy + dz * dz <= 2) m |= 1u << ((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1));
  return m;
}

// Stamps, for the next step, the tiles of the block-wide OR of the cells'
// masks around tile (bx, by, bz) (wrapped; every thread of the block calls
// it); the stamp that first marks a tile for the next step also appends it to
// the next step's list, so every tile is listed once (in no particular order:
// a cell's update depends only on the previous step's values).
template <class Real>
__device__ __forceinline__ void fs_stamp_tiles(const FsArgs<Real> &s, unsigned bx, unsigned by,
                                               unsigned bz, unsigned mask) {
  __shared__ unsigned block_mask;
  if (threadIdx.x == 0) block_mask = 0u;
  __syncthreads();
  mask = __reduce_or_sync(0xffffffffu, mask);
  if ((threadIdx.x & 31u) == 0 && mask) atomicOr(&block_mask, mask);
  __syncthreads();
  const unsigned k = threadIdx.x;
  if (k < 27 && ((block_mask >> k) & 1u)) {
    const unsigned mx = (bx + s.ntx + k % 3 - 1) % s.ntx;
    const unsigned my = (by + s.nty + (k / 3) % 3 - 1) % s.nty;
    const unsigned mz = (bz + s.ntz + k / 9 - 1) % s.ntz;
    const unsigned t = mx + s.ntx * (my + s.nty * mz), v = *s.stamp_ctr + 1u;
    if (atomicExch(s.stamp + t, v) != v) s.next_tiles[atomicAdd(s.next_n_tiles, 1u)] = t;
  }
  __syncthreads();  // block_mask is reset for the next tile only after every read
}

// Cells of this step's active tiles: block b takes list entries b, b +
// gridDim.x, ...; thread k is cell (k % FS_TX, (k / FS_TX) % FS_TY, k /
// (FS_TX FS_TY)) of the tile. cell(n, lx, ly, lz) runs for cells inside the
// lattice; with MARK it returns the cell's tile mask (fs_tile_mask) and the
// tiles of the block's masks are stamped for the next step (the trip count
// is uniform in the block, so every thread reaches the barriers).
template <bool MARK, class Real, class F>
__device__ __forceinline__ void fs_tile_loop(const FsArgs<Real> &s, F &&cell) {
  const unsigned cnt = *s.n_tiles;
  const unsigned tx = threadIdx.x % FS_TX, ty = (threadIdx.x / FS_TX) % FS_TY,
                 tz = threadIdx.x / (FS_TX * FS_TY);
  for (unsigned i = blockIdx.x; i < cnt; i += gridDim.x) {
    const unsigned tile = s.tiles[i];
    const unsigned bx = tile % s.ntx, r = tile / s.ntx, by = r % s.nty, bz = r / s.nty;
    const unsigned x = bx * FS_TX + tx, y = by * FS_TY + ty, z = bz * FS_TZ + tz;
    unsigned mask = 0u;
    if (x < s.a.nx && y < s.a.ny && z < s.a.nz) mask = cell(x + s.a.nx * (y + s.a.ny * z), tx, ty, tz);
    if (MARK) fs_stamp_tiles(s, bx, by, bz, mask);
  }
}

// After initialisation: one block per tile stamps the tiles the first step
// needs around its liquid and interface cells.
template <class Real>
__global__ void __launch_bounds__(FS_BLOCK) fs_seed_kernel(const FsArgs<Real> s) {
  const unsigned tile = blockIdx.x;
  const unsigned bx = tile % s.ntx, r = tile / s.ntx, by = r % s.nty, bz = r / s.nty;
  const unsigned tx = threadIdx.x % FS_TX, ty = (threadIdx.x / FS_TX) % FS_TY,
                 tz = threadIdx.x / (FS_TX * FS_TY);
  const unsigned x = bx * FS_TX + tx, y = by * FS_TY + ty, z = bz * FS_TZ + tz;
  unsigned mask = 0u;
  if (x < s.a.nx && y < s.a.ny && z < s.a.nz) {
    const unsigned n = x + s.a.nx * (y + s.a.ny * z);
    const uint32_t link = s.a.link ? s.a.link[n] : 0u;
    const bool live = !(link >> 31) && s.type_old[n] != CELL_EMPTY;
    mask = fs_tile_mask(tx, ty, tz, live, live);
  }
  fs_stamp_tiles(s, bx, by, bz, mask);
}

// Flowchart step g, Eqs. eq:massmacro, eq:massevol, eq:deltamass:
// m(x, t+1) = m(x, t) + sum_q w (f~_opp(q)(x + c_q) - f~_q(x)), with w = 1 when
// either cell is liquid, (lambda(x) + lambda(x + c_q))/2 between two
// interface cells, and no exchange with empty or solid cells. The colour
// gradient field is the new liquid mass (0 in empty, wall_rho in solid cells).
template <class S>
__global__ void __launch_bounds__(FS_BLOCK) fs_mass_kernel(const FsArgs<typename S::Real> s) {
  using Real = typename S::Real;
  using T = typename S::T;
  const StepArgs<Real> &a = s.a;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *s.any = 0u;
    *s.next_n_tiles = 0u;
    *s.stamp_ctr += 1u;  // read only by the later passes of this step
  }
  fs_tile_loop<false>(s, [&](unsigned n, unsigned, unsigned, unsigned) -> unsigned {
  const uint32_t link = a.link ? __ldg(a.link + n) : 0u;
  if (link >> 31) {
    s.m_new[n] = Real(0);
    s.rhohat_w[n] = a.wall_rho;
    return 0u;
  }
  const uint8_t t = s.type_old[n];
  if (t == CELL_EMPTY) {
    s.m_new[n] = s.m_old[n];
    s.rhohat_w[n] = Real(0);
    return 0u;
  }
  const CellGeo g = cell_geo(n, a.nx, a.ny, a.nz);
  const T *fin = static_cast<const T *>(a.f_in);
  const unsigned N = a.N;
  const Real lx = s.lam[n];
  Real m = s.m_old[n];
  Unroll<1, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const long long y = fs_neighbor<q>(g, n, link, a.f_wall);
    if (y < 0) return;
    const uint8_t ty = s.type_old[y];
    if (ty == CELL_EMPTY) return;
    // the equilibrium weights of q and opp(q) are equal, so deviations subtract
    const Real diff = S::template ld_f<opp(q)>(fin + size_t(opp(q)) * N + y) -
                      S::template ld_f<q>(fin + size_t(q) * N + n);
    const Real w = (t == CELL_INTERFACE && ty == CELL_INTERFACE)
                       ? Real(0.5) * (lx + s.lam[y])
                       : Real(1);
    m += w * diff;
  });
  s.m_new[n] = m;
  s.rhohat_w[n] = m;
  return 0u;
  });
}

// Flowchart steps f, h, e, i for liquid and interface cells: pull-stream with
// bounce-back and, for populations that would come from an empty cell, Eq.
// equilempty: f_q = f^eq_q + f^eq_opp(q) - f~_opp(q)(x) at gas density 1 and
// the cell's own V' (recovered from its post-collision populations; exact
// without Darcy drag); moments, colour gradient, BGK collision with forcing
// and surface tension; then lambda = m / rho and the fill/empty flags.
template <class S>
__global__ void __launch_bounds__(FS_BLOCK, fs_step_blocks<typename S::Real>())
    fs_step_kernel(const FsArgs<typename S::Real> s) {
  using Real = typename S::Real;
  using T = typename S::T;
  static_assert(std::is_same<T, Real>::value, "free surface: storage in the collision type");
  const StepArgs<Real> &a = s.a;
  const unsigned N = a.N;
  fs_tile_loop<false>(s, [&](unsigned n, unsigned, unsigned, unsigned) -> unsigned {
  const uint32_t link = a.link ? __ldg(a.link + n) : 0u;
  const uint8_t t = s.type_old[n];
  s.flag_b[n] = FS_NONE;  // the re-typing pass rewrites it when some cell flags
  if ((link >> 31) || t == CELL_EMPTY) {
    s.flag_a[n] = FS_NONE;
    return 0u;
  }
  const CellGeo g = cell_geo(n, a.nx, a.ny, a.nz);
  const T *__restrict__ fin = static_cast<const T *>(a.f_in);
  T *__restrict__ fout = static_cast<T *>(a.f_out);
  const Real eps = __ldg(a.eps + n);

  // sources that are empty cells
  unsigned from_gas = 0;
  Unroll<1, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    if (fluid_class<q>(g, link, a.f_wall) == PULL_CELL &&
        s.type_old[(long long)n + src_delta<q>(g)] == CELL_EMPTY)
      from_gas |= 1u << q;
  });
  // f^eq_q - w_q at gas density 1 and the cell's own V' (time t), formed per
  // direction from u, 1/eps and u.u (a 19-value array held the kernel at 128
  // registers)
  Real gu0 = Real(0), gu1 = Real(0), gu2 = Real(0), gie = Real(0), guu = Real(0);
  if (from_gas) {
    Real r = Real(0), j0 = Real(0), j1 = Real(0), j2 = Real(0);
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const Real v = S::template ld_f<q>(fin + size_t(q) * N + n);
      r += v;
      if (cx(q)) j0 += Real(cx(q)) * v;
      if (cy(q)) j1 += Real(cy(q)) * v;
      if (cz(q)) j2 += Real(cz(q)) * v;
    });
    const Real ir = Real(1) / (Real(1) + r);
    const Real u0 = j0 * ir - Real(0.5) * eps * a.G[0];
    const Real u1 = j1 * ir - Real(0.5) * eps * a.G[1];
    const Real u2 = j2 * ir - Real(0.5) * eps * a.G[2];
    gu0 = u0;
    gu1 = u1;
    gu2 = u2;
    gie = Real(1) / eps;
    guu = u0 * u0 + u1 * u1 + u2 * u2;
  }
  auto ge = [&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const Real cu = Real(cx(q)) * gu0 + Real(cy(q)) * gu1 + Real(cz(q)) * gu2;
    return wq<Real>(q) * (Real(3) * cu + Real(4.5) * gie * cu * cu - Real(1.5) * gie * guu);
  };
  Real d[Q];
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int cls = fluid_class<q>(g, link, a.f_wall);
    if (cls == PULL_BOUNCE) {
      d[q] = S::template ld_f<opp(q)>(fin + size_t(opp(q)) * N + n);
    } else if ((from_gas >> q) & 1u) {
      d[q] = ge(qc) + ge(std::integral_constant<int, opp(q)>{}) -
             S::template ld_f<opp(q)>(fin + size_t(opp(q)) * N + n);
    } else {
      d[q] = S::template ld_f<q>(fin + size_t(q) * N + (long long)n + src_delta<q>(g));
    }
  });
  Real drho = Real(0), j0 = Real(0), j1 = Real(0), j2 = Real(0);
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    drho += d[q];
    if (cx(q)) j0 += Real(cx(q)) * d[q];
    if (cy(q)) j1 += Real(cy(q)) * d[q];
    if (cz(q)) j2 += Real(cz(q)) * d[q];
  });
  const Real rho = Real(1) + drho;
  const Real irho = Real(1) / rho;
  const Real V[3] = {j0 * irho, j1 * irho, j2 * irho};
  const Real tau = a.tau;
  const Real nu = (tau - Real(0.5)) * Real(1.0 / 3.0);
  FluidCollide<Real> fc;
  fc.F[0] = fc.F[1] = fc.F[2] = Real(0);
  if (a.A != Real(0)) colour_gradient(a.rhohat, n, g, a.f_wall, a.wall_rho, fc.F);
  velocity_solve<KM_NONE>(a.kinv, N, n, eps, nu, V, a.G, fc.Vp, fc.Fe);
  fc.drho = drho;
  fc.rho = rho;
  fc.ie = Real(1) / eps;
  fc.uu = fc.Vp[0] * fc.Vp[0] + fc.Vp[1] * fc.Vp[1] + fc.Vp[2] * fc.Vp[2];
  fc.uF = fc.Vp[0] * fc.Fe[0] + fc.Vp[1] * fc.Fe[1] + fc.Vp[2] * fc.Fe[2];
  fc.itau = Real(1) / tau;
  fc.omt = Real(1) - fc.itau;
  fc.pre = rho * (Real(1) - Real(0.5) * fc.itau);
  fc.Fn = sqrt(fc.F[0] * fc.F[0] + fc.F[1] * fc.F[1] + fc.F[2] * fc.F[2]);
  fc.st = (a.A != Real(0)) && fc.Fn > st_threshold<Real>();
  fc.stc = fc.st ? a.A * eps * tau : Real(0);
  fc.iFn = fc.st ? Real(1) / fc.Fn : Real(0);
  fc.fold(Real(1), Real(0));
  // the post-collision density, summed from the stored values in direction
  // order (as the liquid fraction and a filled cell's excess mass need it)
  Real rp = Real(0);
  Unroll<0, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const Real v = fc.template post<q>(d[q]);
    S::template st_f<q>(fout + size_t(q) * N + n, v);
    rp += v;  // the stored value: FP32 / FP64 storage holds the collision type
  });
  s.rho_post[n] = Real(1) + rp;
  write_fields(a.fields, N, n, rho, fc.Vp, Real(0), nu);
  // the moments a new interface cell averages: it was empty, so each of its
  // live neighbours pulled from it in this pass
  if (from_gas) {
    s.mom[n] = rho;
    s.mom[size_t(N) + n] = fc.Vp[0];
    s.mom[2 * size_t(N) + n] = fc.Vp[1];
    s.mom[3 * size_t(N) + n] = fc.Vp[2];
  }
  // flowchart step j, candidates: lambda > 1 + 1e-3 fills, lambda < -1e-3 empties
  uint8_t flag = FS_NONE;
  if (t == CELL_INTERFACE) {
    const Real lam = s.m_new[n] / rho;
    if (lam > Real(1.001))
      flag = FS_FILL;
    else if (lam < Real(-0.001))
      flag = FS_EMPTYING;
  }
  s.flag_a[n] = flag;
  if (flag) atomicOr(s.any, 1u);
  return 0u;
  });
}

// Whether an emptying cell y is next to a filling one (then it stays an
// interface cell), from the step's flags.
template <class Real>
__device__ __forceinline__ bool fs_near_fill(const FsArgs<Real> &s, long long y) {
  const StepArgs<Real> &a = s.a;
  const uint32_t link = a.link ? a.link[y] : 0u;
  const CellGeo g = cell_geo(unsigned(y), a.nx, a.ny, a.nz);
  bool near = false;
  Unroll<1, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const long long y2 = fs_neighbor<q>(g, unsigned(y), link, a.f_wall);
    if (y2 >= 0 && s.flag_a[y2] == FS_FILL) near = true;
  });
  return near;
}

// New cell types, with the cancellation of an emptying cell next to a filling
// one folded in (it reads the step's flags two links away): filled -> liquid,
// emptied -> empty, empty next to a filled cell -> interface (flagged
// FS_NEWCELL), liquid next to an emptied cell -> interface. flag_b gets each
// cell's settled flag.
template <class Real>
__global__ void __launch_bounds__(FS_BLOCK) fs_retype_kernel(const FsArgs<Real> s) {
  const StepArgs<Real> &a = s.a;
  fs_tile_loop<false>(s, [&](unsigned n, unsigned, unsigned, unsigned) -> unsigned {
  uint8_t t = s.type_old[n];
  const uint32_t link = a.link ? a.link[n] : 0u;
  if (*s.any != 0u && !(link >> 31)) {
    uint8_t f = s.flag_a[n];
    if (f == FS_EMPTYING && fs_near_fill(s, n)) f = FS_NONE;
    if (f == FS_FILL) {
      t = CELL_LIQUID;
    } else if (f == FS_EMPTYING) {
      t = CELL_EMPTY;
    } else if (t == CELL_EMPTY || t == CELL_LIQUID) {
      const CellGeo g = cell_geo(n, a.nx, a.ny, a.nz);
      const bool empty = t == CELL_EMPTY;
      bool hit = false;
      Unroll<1, Q>::run([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const long long y = fs_neighbor<q>(g, n, link, a.f_wall);
        if (y < 0) return;
        const uint8_t fy = s.flag_a[y];
        if (empty ? fy == FS_FILL : (fy == FS_EMPTYING && !fs_near_fill(s, y))) hit = true;
      });
      if (hit) {
        t = CELL_INTERFACE;
        if (empty) f = FS_NEWCELL;
      }
    }
    s.flag_b[n] = f;
  }
  s.type_new[n] = t;
  return 0u;
  });
}

// New interface cells take f = f^eq(mean rho, mean V') of their liquid and
// interface neighbours that are not new themselves (hydrodynamic
// equilibrium, no mass); filled and emptied cells hand their excess mass (m -
// rho, or m) in equal shares to the neighbours that are interface cells after
// the re-typing (they keep it when there are none).
template <class S>
__global__ void __launch_bounds__(FS_BLOCK) fs_newcell_kernel(const FsArgs<typename S::Real> s) {
  using Real = typename S::Real;
  using T = typename S::T;
  const StepArgs<Real> &a = s.a;
  const unsigned N = a.N;
  if (*s.any == 0u) return;
  fs_tile_loop<false>(s, [&](unsigned n, unsigned, unsigned, unsigned) -> unsigned {
  const uint8_t f = s.flag_b[n];
  if (f == FS_NONE) return 0u;
  const uint32_t link = a.link ? a.link[n] : 0u;
  const CellGeo g = cell_geo(n, a.nx, a.ny, a.nz);
  if (f == FS_NEWCELL) {
    // density and V' of each neighbour as its collision in this step left
    // them (its post-collision populations carry the same moments: the
    // collision conserves mass, and without Darcy drag their momentum is
    // rho (V' + eps G / 2)); the loads of all neighbours are in flight together
    Real rs = Real(0), u0 = Real(0), u1 = Real(0), u2 = Real(0);
    int cnt = 0;
    Unroll<1, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const long long y = fs_neighbor<q>(g, n, link, a.f_wall);
      if (y < 0) return;
      const uint8_t ty = s.type_new[y];
      if ((ty != CELL_LIQUID && ty != CELL_INTERFACE) || s.flag_b[y] == FS_NEWCELL) return;
      rs += s.mom[y];
      u0 += s.mom[size_t(N) + y];
      u1 += s.mom[2 * size_t(N) + y];
      u2 += s.mom[3 * size_t(N) + y];
      ++cnt;
    });
    const Real ic = Real(1) / Real(cnt > 0 ? cnt : 1);
    const Real r = cnt > 0 ? rs * ic : Real(1);
    const Real u[3] = {u0 * ic, u1 * ic, u2 * ic};
    const Real eps = a.eps[n];
    const Real ie = Real(1) / eps, uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T *fout = static_cast<T *>(a.f_out);
    Real rp = Real(0);
    Unroll<0, Q>::run([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const Real cu = Real(cx(q)) * u[0] + Real(cy(q)) * u[1] + Real(cz(q)) * u[2];
      const Real dev = wq<Real>(q) * ((r - Real(1)) +
                                      r * (Real(3) * cu + Real(4.5) * ie * cu * cu -
                                           Real(1.5) * ie * uu));
      S::template st_f<q>(fout + size_t(q) * N + n, dev);
      rp += dev;
    });
    s.rho_post[n] = Real(1) + rp;  // the density of the stored populations, for lambda
    write_fields(a.fields, N, n, r, u, Real(0), (a.tau - Real(0.5)) / Real(3));
    return 0u;
  }
  int cnt = 0;
  Unroll<1, Q>::run([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const long long y = fs_neighbor<q>(g, n, link, a.f_wall);
    if (y >= 0 && s.type_new[y] == CELL_INTERFACE) ++cnt;
  });
  // a filled cell keeps m = rho: its post-collision density in the collision
  // type (the exported field is float)
  Real share = Real(0);
  if (cnt > 0) {
    const Real m = s.m_new[n];
    const Real excess = (f == FS_FILL) ? m - s.rho_post[n] : m;
    share = excess / Real(cnt);
    s.m_new[n] = m - excess;
  }
  s.share[n] = share;
  return 0u;
  });
}

// Excess mass arrives at interface cells; types settle; lambda = m / rho;
// the next step's tiles are stamped and listed.
template <class S>
__global__ void __launch_bounds__(FS_BLOCK) fs_finish_kernel(const FsArgs<typename S::Real> s) {
  using Real = typename S::Real;
  const StepArgs<Real> &a = s.a;
  const unsigned N = a.N;
  fs_tile_loop<true>(s, [&](unsigned n, unsigned lx, unsigned ly, unsigned lz) -> unsigned {
  const uint32_t link = a.link ? a.link[n] : 0u;
  if (link >> 31) {
    s.lam[n] = Real(0);
    return 0u;
  }
  const uint8_t tn = s.type_new[n];
  Real m = s.m_new[n];
  if (*s.any != 0u) {
    if (tn == CELL_INTERFACE) {
      const CellGeo g = cell_geo(n, a.nx, a.ny, a.nz);
      Unroll<1, Q>::run([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const long long y = fs_neighbor<q>(g, n, link, a.f_wall);
        if (y < 0) return;
        const uint8_t fy = s.flag_b[y];
        if (fy == FS_FILL || fy == FS_EMPTYING) m += s.share[y];
      });
      s.m_new[n] = m;
    }
    if (tn == CELL_EMPTY && s.flag_b[n] == FS_EMPTYING) zero_fields(a.fields, N, n);
  }
  s.lam[n] = tn == CELL_LIQUID ? Real(1) : (tn == CELL_EMPTY ? Real(0) : m / s.rho_post[n]);
  // both buffers of the type and the mass agree after the step, so a cell
  // whose tile leaves the list keeps the same values under either parity
  s.type_old[n] = tn;
  s.m_old[n] = m;
  // the next step needs every cell within one link of a liquid or interface
  // cell, and each cell flagged in this step (its flags are cleared then)
  return fs_tile_mask(lx, ly, lz, s.flag_b[n] != FS_NONE, tn != CELL_EMPTY);
  });
}

}  // namespace lbgb
