/*
 * Oracle for the porous-media lattice-Boltzmann scheme of Mendoza, Wittel and
 * Herrmann (arXiv:0912.4230). TEST INFRASTRUCTURE ONLY: see lb_oracle.h.
 *
 * Everything is FP64 and cell by cell, in the order of the paper's flowchart
 * (Section 4, Fig. flowchart): t = t+1, stream f and h (step f), stream the
 * liquid mass (step g), moments (step h), colour gradient (step e), collide
 * (step i), re-type free-surface cells (step j). Cells are visited in index
 * order; OpenMP only splits loops whose iterations write disjoint cells, and
 * every sum across cells is taken serially in index order.
 *
 * Readings of places where the paper is silent or garbled are marked
 * "Reading:" in the comments; each one is also listed in the design notes.
 */
#include "lb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* ------------------------------------------------------------------------ */
/* D3Q19 velocity set (Section 2.1, Fig. d3q19; weights after Eq. equilc2).  */
/* ------------------------------------------------------------------------ */

static int CV[Q][3];
static double WT[Q];
static int OPP[Q];
static int table_ready = 0;

/* Reading (the figure is not available): q = 1 + 6p + (i-1) for orientation
 * i = 1..6 in reference plane p = 0 (x-y), 1 (y-z), 2 (z-x). Orientations
 * 1..4 are the plane's diagonals, counter-clockwise from (+first, +second)
 * axis, weight 1/36; orientations 5, 6 are +/- the plane's first axis, weight
 * 1/18; the rest vector q = 0 has weight 1/3. */
static void make_velocity_set(void)
{
  static const int plane_axes[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  static const int diag[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
  if (table_ready) return;
  memset(CV, 0, sizeof CV);
  WT[0] = 1.0 / 3.0;
  for (int p = 0; p < 3; p++) {
    int a0 = plane_axes[p][0], a1 = plane_axes[p][1];
    for (int i = 1; i <= 6; i++) {
      int q = 1 + 6 * p + (i - 1);
      if (i <= 4) {
        CV[q][a0] = diag[i - 1][0];
        CV[q][a1] = diag[i - 1][1];
        WT[q] = 1.0 / 36.0;
      } else {
        CV[q][a0] = (i == 5) ? 1 : -1;
        WT[q] = 1.0 / 18.0;
      }
    }
  }
  /* opposite direction by exhaustive search */
  for (int q = 0; q < Q; q++)
    for (int r = 0; r < Q; r++)
      if (CV[r][0] == -CV[q][0] && CV[r][1] == -CV[q][1] && CV[r][2] == -CV[q][2])
        OPP[q] = r;
  table_ready = 1;
}

void orc_velocity_set(int32_t *c, double *w, int32_t *opp)
{
  make_velocity_set();
  for (int q = 0; q < Q; q++) {
    for (int a = 0; a < 3; a++) c[3 * q + a] = CV[q][a];
    w[q] = WT[q];
    opp[q] = OPP[q];
  }
}

static double dot3(const double *a, const double *b)
{
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static double cdot(int q, const double *v)
{
  return CV[q][0] * v[0] + CV[q][1] * v[1] + CV[q][2] * v[2];
}

/* Inverse of a general 3x3 matrix (row-major) by the adjugate. */
static void inv3(const double *M, double *R)
{
  double a = M[0], b = M[1], c = M[2];
  double d = M[3], e = M[4], f = M[5];
  double g = M[6], h = M[7], i = M[8];
  double A = e * i - f * h, B = -(d * i - f * g), Cc = d * h - e * g;
  double det = a * A + b * B + c * Cc;
  R[0] = A / det;
  R[1] = -(b * i - c * h) / det;
  R[2] = (b * f - c * e) / det;
  R[3] = B / det;
  R[4] = (a * i - c * g) / det;
  R[5] = -(a * f - c * d) / det;
  R[6] = Cc / det;
  R[7] = -(a * h - b * g) / det;
  R[8] = (a * e - b * d) / det;
}

/* ------------------------------------------------------------------------ */
/* Single-cell pieces of the model (Section 2).                              */
/* ------------------------------------------------------------------------ */

/* Equilibrium of the fluid populations, Eqs. equilc1 and equilc2, including
 * the surface-tension terms. Reading: where |F| vanishes the surface-tension
 * term (which contains (c.F)^2/|F|) is taken as zero. */
void orc_feq(double rho, const double *u, double eps, double tau, double A,
             const double *F, double *out)
{
  make_velocity_set();
  double uu = dot3(u, u);
  double Fn = sqrt(dot3(F, F));
  int st = (A != 0.0 && Fn > 1e-30);
  out[0] = WT[0] * rho * (1.0 - 1.5 / eps * uu) + (st ? A * eps * tau * WT[0] * Fn : 0.0);
  for (int q = 1; q < Q; q++) {
    double cu = cdot(q, u);
    double hydro = WT[q] * rho * (1.0 + 3.0 * cu + 4.5 / eps * cu * cu - 1.5 / eps * uu);
    double surf = 0.0;
    if (st) {
      double cF = cdot(q, F);
      surf = WT[q] * A * eps * tau * (cF * cF / Fn - Fn);
    }
    out[q] = hydro + surf;
  }
}

/* Forcing terms T_q and T_0, Eq. coeffforce1. Reading: as printed the terms
 * carry neither the weight w_q nor the density; they are taken with the
 * factor w_q*rho of the cited forcing scheme (Guo et al.), without which
 * sum_q T_q would not vanish and mass would not be conserved. */
void orc_forcing(double rho, double tau, double eps, const double *u,
                 const double *Fext, double *out)
{
  make_velocity_set();
  double pre = 1.0 - 0.5 / tau;
  double uF = dot3(u, Fext);
  for (int q = 0; q < Q; q++) {
    double cu = cdot(q, u), cF = cdot(q, Fext);
    out[q] = WT[q] * rho * pre * (3.0 * cF + 9.0 / eps * cu * cF - 3.0 / eps * uF);
  }
}

/* Velocity correction and Darcy force, Eqs. forcement, expandV, expandVsub.
 * Substituting Eq. forcement into Eq. expandV gives
 *   (I + (eps nu / 2) K^-1) V' = V + (eps / 2) G,
 * so the reading is V' = Lambda^-1 (V + eps G / 2) (the printed Eq. expandVsub
 * drops the eps in front of G). Kinv9 = NULL means K^-1 = 0.
 *
 * Forchheimer drag (cF != 0; reading R21, the paper names the term but gives
 * no equation): the porous-flow model the paper builds on (Guo and Zhao) adds
 * -eps F_eps |V'| K^-1/2 V' to the force, F_eps = cF 1.75 / sqrt(150 eps^3)
 * (Ergun), with K^-1/2 = diag(sqrt(K^-1_ii)) for a diagonal K. With the same
 * half-force velocity V' = V + F^ext / 2 this gives, axis by axis,
 *   V'_i (1 + eps nu k_i / 2 + eps F_eps sqrt(k_i) s / 2) = V_i + eps G_i / 2,
 * with s = |V'|. The right-hand side of s = |V'(s)| decreases in s, so the
 * root is unique in [0, |V'(0)|]; it is found by bisection to the last bit. */
void orc_velocity_solve(const double *V, double eps, double nu,
                        const double *Kinv9, const double *G, double cF,
                        double *Vp, double *Fext)
{
  double r[3];
  for (int i = 0; i < 3; i++) r[i] = V[i] + 0.5 * eps * G[i];
  if (cF != 0.0 && Kinv9) {
    double Fe = cF * 1.75 / sqrt(150.0 * eps * eps * eps);
    double a[3], b[3], k[3];
    for (int i = 0; i < 3; i++) {
      k[i] = Kinv9[4 * i];  /* diagonal entries */
      a[i] = 1.0 + 0.5 * eps * nu * k[i];
      b[i] = 0.5 * eps * Fe * sqrt(k[i]);
    }
    double lo = 0.0, hi = 0.0;
    for (int i = 0; i < 3; i++) hi += (r[i] / a[i]) * (r[i] / a[i]);
    hi = sqrt(hi);
    for (int it = 0; it < 200; it++) {
      double mid = 0.5 * (lo + hi), m2 = 0.0;
      for (int i = 0; i < 3; i++) {
        double v = r[i] / (a[i] + b[i] * mid);
        m2 += v * v;
      }
      if (sqrt(m2) > mid) lo = mid; else hi = mid;
    }
    double sv = 0.5 * (lo + hi);
    for (int i = 0; i < 3; i++) Vp[i] = r[i] / (a[i] + b[i] * sv);
    double speed = sqrt(dot3(Vp, Vp));
    for (int i = 0; i < 3; i++)
      Fext[i] = -eps * nu * k[i] * Vp[i] - eps * Fe * sqrt(k[i]) * speed * Vp[i] + eps * G[i];
    return;
  }
  double L[9], Li[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      L[3 * i + j] = (i == j ? 1.0 : 0.0) + (Kinv9 ? 0.5 * eps * nu * Kinv9[3 * i + j] : 0.0);
  inv3(L, Li);
  for (int i = 0; i < 3; i++)
    Vp[i] = Li[3 * i + 0] * r[0] + Li[3 * i + 1] * r[1] + Li[3 * i + 2] * r[2];
  for (int i = 0; i < 3; i++) {
    double kv = 0.0;
    if (Kinv9)
      kv = Kinv9[3 * i + 0] * Vp[0] + Kinv9[3 * i + 1] * Vp[1] + Kinv9[3 * i + 2] * Vp[2];
    Fext[i] = -eps * nu * kv + eps * G[i];
  }
}

/* Solute equilibrium, Eq. equild. */
void orc_heq(double eps, double Cc, const double *Vstar, double *out)
{
  make_velocity_set();
  for (int q = 0; q < Q; q++) out[q] = WT[q] * eps * Cc * (1.0 + 3.0 * cdot(q, Vstar));
}

/* Relaxation time from the viscosity law. nu = (tau - 1/2)/3 (Section 2,
 * after Eq. eqsurftens). Law 2 is Eq. nuall; reading: t is the step index
 * after the increment of flowchart step d (t = 0 at initialisation). */
double orc_tau_of(const orc_params *p, double Cc, int64_t t)
{
  if (p->visc_law == 1) {
    double cl = Cc < 0.0 ? 0.0 : (Cc > 1.0 ? 1.0 : Cc);
    return p->tau0 + (p->tau1 - p->tau0) * cl;
  }
  if (p->visc_law == 2) {
    double nu = p->nu_g * (1.0 + p->a * exp(p->alpha * (double)t)) * exp(p->beta * (1.0 - Cc));
    return 3.0 * nu + 0.5;
  }
  return p->tau;
}

/* Hydrodynamic part of Eq. equilc1/equilc2 (no surface-tension term), used by
 * the free-surface reconstruction and the initialisation of new interface
 * cells. */
static void feq_hydro(double rho, const double *u, double eps, double *out)
{
  double zero[3] = {0.0, 0.0, 0.0};
  orc_feq(rho, u, eps, 1.0, 0.0, zero, out);
}

/* ------------------------------------------------------------------------ */
/* Lattice state.                                                           */
/* ------------------------------------------------------------------------ */

struct orc {
  orc_params p;
  int64_t N;
  double *f, *fn, *fs; /* post-collision at t, at t+1, and post-stream scratch */
  double *h, *hn, *hs;
  double *eps;
  double *Kinv;        /* 9 per cell, NULL = K infinite */
  double *geps;        /* grad(eps)/eps, 3 per cell */
  uint8_t *solid;
  uint8_t *type, *ntype, *flag;
  double *m, *mn, *lam;
  double *rhohat;
  double *out_rho, *out_u, *out_C, *out_nu;
  double *cell_in, *cell_out; /* per-cell solute flux of the current step */
  int64_t t;
  int S;               /* solute species (0 without the solute lattice) */
  double flux_in[ORC_MAX_SPECIES], flux_out[ORC_MAX_SPECIES];
};

static int64_t cell_index(const orc *o, int x, int y, int z)
{
  return (int64_t)x + (int64_t)o->p.nx * ((int64_t)y + (int64_t)o->p.ny * z);
}

static void cell_coords(const orc *o, int64_t n, int *x, int *y, int *z)
{
  *x = (int)(n % o->p.nx);
  *y = (int)((n / o->p.nx) % o->p.ny);
  *z = (int)(n / ((int64_t)o->p.nx * o->p.ny));
}

/* Where the population arriving at cell (x,y,z) along c_q comes from during
 * the stream step (Eq. lbe2: the cell at x - c_q feeds f_q at x). Periodic
 * faces wrap. Reading (walls): a face of kind WALL, or a solid source cell,
 * gives halfway bounce-back. Open faces (readings R9, R23): a population that
 * enters through a face of kind INLET, OUTLET, PRESSURE or VELOCITY takes that
 * face's rule. Precedence when a diagonal leaves through two faces: WALL >
 * VELOCITY > PRESSURE > INLET > OUTLET, and between two faces of one kind the
 * one on the lower axis. Returns the source index or an ORC_SRC_ class; *face
 * (may be NULL) receives 2 axis + side of the deciding face. */
static int64_t pull_source(const orc *o, const int32_t kinds[3][2], int x, int y,
                           int z, int q, int *face)
{
  int c[3] = {x - CV[q][0], y - CV[q][1], z - CV[q][2]};
  int n[3] = {o->p.nx, o->p.ny, o->p.nz};
  /* rank of each kind in the precedence order (0 = none) and its face */
  static const int rank[6] = {0, 5, 2, 1, 3, 4};
  static const int64_t cls[6] = {0, ORC_SRC_BOUNCE, ORC_SRC_INLET, ORC_SRC_OUTLET,
                                 ORC_SRC_PRESSURE, ORC_SRC_VELOCITY};
  int best = 0, best_face = -1;
  for (int a = 0; a < 3; a++) {
    if (c[a] >= 0 && c[a] < n[a]) continue;
    int side = c[a] < 0 ? 0 : 1;
    int k = kinds[a][side];
    if (k == ORC_PERIODIC) {
      c[a] = (c[a] + n[a]) % n[a];
      continue;
    }
    if (best == 0 || rank[k] > rank[best]) {
      best = k;
      best_face = 2 * a + side;
    }
  }
  if (face) *face = best_face;
  if (best != 0) return cls[best];
  int64_t s = cell_index(o, c[0], c[1], c[2]);
  if (o->solid[s]) return ORC_SRC_BOUNCE;
  return s;
}

/* The neighbour x + c_q; -1 when the step leaves through a non-periodic face. */
static int64_t neighbor(const orc *o, const int32_t kinds[3][2], int x, int y, int z,
                        int q)
{
  int c[3] = {x + CV[q][0], y + CV[q][1], z + CV[q][2]};
  int n[3] = {o->p.nx, o->p.ny, o->p.nz};
  for (int a = 0; a < 3; a++) {
    if (c[a] >= 0 && c[a] < n[a]) continue;
    if (kinds[a][c[a] < 0 ? 0 : 1] != ORC_PERIODIC) return -1;
    c[a] = (c[a] + n[a]) % n[a];
  }
  return cell_index(o, c[0], c[1], c[2]);
}

/* fluid faces: PERIODIC, WALL, PRESSURE, VELOCITY; solute faces: PERIODIC,
 * WALL, INLET, OUTLET; a pair of opposite faces is periodic on both sides or
 * on neither */
static int valid_faces(const int32_t k[3][2], int fluid)
{
  for (int a = 0; a < 3; a++) {
    for (int s = 0; s < 2; s++) {
      int v = k[a][s];
      if (fluid ? !(v == ORC_PERIODIC || v == ORC_WALL || v == ORC_PRESSURE || v == ORC_VELOCITY)
                : (v < 0 || v > 3))
        return 0;
    }
    if ((k[a][0] == ORC_PERIODIC) != (k[a][1] == ORC_PERIODIC)) return 0;
  }
  return 1;
}

static void *zalloc(size_t n) { return calloc(n ? n : 1, 1); }

void orc_destroy(orc *o)
{
  if (!o) return;
  double *d[] = {o->f, o->fn, o->fs, o->h, o->hn, o->hs, o->eps, o->Kinv, o->geps,
                 o->m, o->mn, o->lam, o->rhohat, o->out_rho, o->out_u, o->out_C,
                 o->out_nu, o->cell_in, o->cell_out};
  for (size_t i = 0; i < sizeof d / sizeof d[0]; i++) free(d[i]);
  free(o->solid);
  free(o->type);
  free(o->ntype);
  free(o->flag);
  free(o);
}

/* Cholesky test for a symmetric 3x3 matrix (positive definiteness). */
static int spd3(const double *M)
{
  double l00 = M[0];
  if (!(l00 > 0)) return 0;
  l00 = sqrt(l00);
  double l10 = M[3] / l00, l20 = M[6] / l00;
  double d1 = M[4] - l10 * l10;
  if (!(d1 > 0)) return 0;
  double l11 = sqrt(d1);
  double l21 = (M[7] - l20 * l10) / l11;
  double d2 = M[8] - l20 * l20 - l21 * l21;
  return d2 > 0;
}

orc *orc_create(const orc_params *p, const double *eps, const double *K6,
                const uint8_t *solid)
{
  make_velocity_set();
  if (!p || !eps || !solid) return NULL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
  if (!valid_faces(p->bc, 1) || !valid_faces(p->sbc, 0)) return NULL;
  for (int a = 0; a < 3; a++)
    for (int s = 0; s < 2; s++)
      if (p->bc[a][s] == ORC_WALL && p->sbc[a][s] != ORC_WALL) return NULL;
  if (p->visc_law == 0 && !(p->tau > 0.5)) return NULL;
  if (p->visc_law == 1 && !(p->tau0 > 0.5 && p->tau1 > 0.5)) return NULL;
  if (p->visc_law == 2 && !(p->nu_g > 0)) return NULL;
  if (p->visc_law < 0 || p->visc_law > 2) return NULL;
  if (p->visc_law != 0 && !p->solute) return NULL;
  if (p->solute && !(p->tau_D > 0.5)) return NULL;
  if (p->free_surface && (p->solute || K6)) return NULL;
  if (p->forchheimer < 0.0) return NULL;
  {
    int open_fluid = 0;
    for (int a = 0; a < 3; a++)
      for (int s = 0; s < 2; s++)
        if (p->bc[a][s] == ORC_PRESSURE || p->bc[a][s] == ORC_VELOCITY) open_fluid = 1;
    if (open_fluid && (p->free_surface || p->A != 0.0)) return NULL;
  }
  if (p->forchheimer != 0.0 && K6) {  /* the Forchheimer reading needs a diagonal K */
    int64_t N0 = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t n = 0; n < N0; n++)
      if (K6[6 * n + 3] != 0.0 || K6[6 * n + 4] != 0.0 || K6[6 * n + 5] != 0.0) return NULL;
  }

  if (p->species < 0 || p->species > ORC_MAX_SPECIES) return NULL;
  if (p->species > 1 && !p->solute) return NULL;
  for (int sp = 1; sp < p->species; sp++)
    if (!(p->species_tau_D[sp] > 0.5)) return NULL;

  orc *o = (orc *)zalloc(sizeof(orc));
  o->p = *p;
  int64_t N = (int64_t)p->nx * p->ny * p->nz;
  o->N = N;
  o->S = p->solute ? (p->species > 1 ? p->species : 1) : 0;
  int S1 = o->S > 1 ? o->S : 1;
#ifdef _OPENMP
  if (p->threads > 0) omp_set_num_threads(p->threads);
#endif
  size_t nq = (size_t)N * Q * sizeof(double);
  o->f = zalloc(nq);
  o->fn = zalloc(nq);
  o->fs = zalloc(nq);
  if (p->solute) {
    o->h = zalloc(o->S * nq);
    o->hn = zalloc(o->S * nq);
    o->hs = zalloc(o->S * nq);
  }
  o->eps = zalloc(N * sizeof(double));
  o->geps = zalloc(3 * N * sizeof(double));
  o->solid = zalloc(N);
  o->type = zalloc(N);
  o->ntype = zalloc(N);
  o->flag = zalloc(N);
  o->m = zalloc(N * sizeof(double));
  o->mn = zalloc(N * sizeof(double));
  o->lam = zalloc(N * sizeof(double));
  o->rhohat = zalloc(N * sizeof(double));
  o->out_rho = zalloc(N * sizeof(double));
  o->out_u = zalloc(3 * N * sizeof(double));
  o->out_C = zalloc(S1 * N * sizeof(double));
  o->out_nu = zalloc(N * sizeof(double));
  o->cell_in = zalloc(S1 * N * sizeof(double));
  o->cell_out = zalloc(S1 * N * sizeof(double));
  memcpy(o->solid, solid, N);
  for (int64_t n = 0; n < N; n++) {
    o->eps[n] = eps[n];
    if (!solid[n] && !(eps[n] > 0.0 && eps[n] <= 1.0)) {
      orc_destroy(o);
      return NULL;
    }
  }
  if (K6) {
    o->Kinv = zalloc(9 * N * sizeof(double));
    for (int64_t n = 0; n < N; n++) {
      const double *k = K6 + 6 * n; /* xx, yy, zz, xy, yz, zx */
      double M[9] = {k[0], k[3], k[5], k[3], k[1], k[4], k[5], k[4], k[2]};
      if (solid[n]) continue;
      if (!spd3(M)) {
        orc_destroy(o);
        return NULL;
      }
      inv3(M, o->Kinv + 9 * n);
    }
  }
  /* grad(eps)/eps for V* = V' + D grad(eps)/eps (Eq. equild). Reading: the
   * isotropic lattice gradient 3 sum_q w_q eps(x + c_q) c_q on the solute
   * lattice's topology; a solid or out-of-box neighbour contributes eps(x). */
  for (int64_t n = 0; n < N; n++) {
    int x, y, z;
    cell_coords(o, n, &x, &y, &z);
    double g[3] = {0, 0, 0};
    for (int q = 1; q < Q; q++) {
      int64_t b = neighbor(o, p->sbc, x, y, z, q);
      double e = (b < 0 || solid[b]) ? o->eps[n] : o->eps[b];
      for (int a = 0; a < 3; a++) g[a] += 3.0 * WT[q] * e * CV[q][a];
    }
    for (int a = 0; a < 3; a++) o->geps[3 * n + a] = g[a] / o->eps[n];
  }
  return o;
}

/* Species s >= 1 carry their own relaxation time and inlet concentration
 * (reading R24); D = (tau_D - 1/2) / 3 (Section 2.2). */
static double tau_D_of(const orc *o, int s) { return s ? o->p.species_tau_D[s] : o->p.tau_D; }
static double C_in_of(const orc *o, int s) { return s ? o->p.species_C_in[s] : o->p.C_in; }
static double diffusivity_of(const orc *o, int s) { return (tau_D_of(o, s) - 0.5) / 3.0; }
static double diffusivity(const orc *o) { return diffusivity_of(o, 0); }

/* Colour gradient F = sum_q rhohat(x + c_q) c_q (Eq. macros, second part).
 * Reading: the sum is unweighted as printed; a solid neighbour, or a step out
 * through a wall face, contributes wall_rho. */
static void colour_gradient(const orc *o, int64_t n, double *F)
{
  int x, y, z;
  cell_coords(o, n, &x, &y, &z);
  F[0] = F[1] = F[2] = 0.0;
  for (int q = 1; q < Q; q++) {
    int64_t b = neighbor(o, o->p.bc, x, y, z, q);
    double r = (b < 0 || o->solid[b]) ? o->p.wall_rho : o->rhohat[b];
    for (int a = 0; a < 3; a++) F[a] += r * CV[q][a];
  }
}

/* V' of a cell recovered from its post-collision populations (free surface
 * only, where K^-1 = 0): sum_q f~_q c_q / rho = V' + eps G / 2 exactly. */
static void post_collision_velocity(const orc *o, const double *f, int64_t n,
                                    double *rho, double *u)
{
  double r = 0, j[3] = {0, 0, 0};
  for (int q = 0; q < Q; q++) {
    double v = f[(int64_t)q * o->N + n];
    r += v;
    for (int a = 0; a < 3; a++) j[a] += v * CV[q][a];
  }
  *rho = r;
  for (int a = 0; a < 3; a++) u[a] = j[a] / r - 0.5 * o->eps[n] * o->p.G[a];
}

int orc_init(orc *o, const double *rho0, const double *u0, const double *C0,
             const uint8_t *type, const double *lambda0, const double *f_scale)
{
  if (!o || !rho0 || !u0) return -1;
  if (o->p.solute && !C0) return -1;
  if (o->p.free_surface && !type) return -1;
  int64_t N = o->N;
  o->t = 0;
  for (int sp = 0; sp < ORC_MAX_SPECIES; sp++) o->flux_in[sp] = o->flux_out[sp] = 0.0;
  /* flowchart steps a and b: fields, cell types and cell masses */
  for (int64_t n = 0; n < N; n++) {
    o->type[n] = o->p.free_surface ? type[n] : ORC_LIQUID;
    if (o->solid[n]) {
      o->m[n] = o->lam[n] = 0.0;
      continue;
    }
    double lam = 1.0;
    if (o->type[n] == ORC_INTERFACE) lam = lambda0 ? lambda0[n] : 0.5;
    if (o->type[n] == ORC_EMPTY) lam = 0.0;
    o->lam[n] = lam;
    o->m[n] = lam * rho0[n];
  }
  for (int64_t n = 0; n < N; n++) {
    if (o->solid[n])
      o->rhohat[n] = o->p.wall_rho;
    else if (o->p.free_surface)
      o->rhohat[n] = o->m[n];
    else
      o->rhohat[n] = rho0[n];
  }
  /* flowchart step c: f = f^eq, h = h^eq */
  memset(o->f, 0, (size_t)N * Q * sizeof(double));
  if (o->p.solute) memset(o->h, 0, (size_t)o->S * N * Q * sizeof(double));
  for (int sp = 1; sp < o->S; sp++)
    for (int64_t n = 0; n < N; n++) o->out_C[sp * N + n] = 0.0;
  for (int64_t n = 0; n < N; n++) {
    o->out_rho[n] = o->out_C[n] = o->out_nu[n] = 0.0;
    o->out_u[3 * n] = o->out_u[3 * n + 1] = o->out_u[3 * n + 2] = 0.0;
    if (o->solid[n] || o->type[n] == ORC_EMPTY) continue;
    double Cc = o->p.solute ? C0[n] : 0.0;
    double tau = orc_tau_of(&o->p, Cc, 0);
    double F[3] = {0, 0, 0}, fe[Q];
    if (o->p.A != 0.0) colour_gradient(o, n, F);
    orc_feq(rho0[n], u0 + 3 * n, o->eps[n], tau, o->p.A, F, fe);
    for (int q = 0; q < Q; q++)
      o->f[(int64_t)q * N + n] = fe[q] * (f_scale ? f_scale[(int64_t)q * N + n] : 1.0);
    for (int sp = 0; sp < o->S; sp++) {
      double Vs[3], he[Q], Cs = C0[sp * N + n], D = diffusivity_of(o, sp);
      for (int a = 0; a < 3; a++) Vs[a] = u0[3 * n + a] + D * o->geps[3 * n + a];
      orc_heq(o->eps[n], Cs, Vs, he);
      for (int q = 0; q < Q; q++) o->h[((int64_t)sp * Q + q) * N + n] = he[q];
      o->out_C[sp * N + n] = Cs;
    }
    o->out_rho[n] = rho0[n];
    for (int a = 0; a < 3; a++) o->out_u[3 * n + a] = u0[3 * n + a];
    o->out_nu[n] = (tau - 0.5) / 3.0;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One time step.                                                            */
/* ------------------------------------------------------------------------ */

static int active(const orc *o, int64_t n)
{
  return !o->solid[n] && o->type[n] != ORC_EMPTY;
}

/* Density and velocity j / rho of the cell's own post-collision populations
 * (the previous step's output buffer). */
static void post_collision_moments(const orc *o, int64_t n, double *rho, double *u)
{
  double r = 0, j[3] = {0, 0, 0};
  for (int q = 0; q < Q; q++) {
    double v = o->f[(int64_t)q * o->N + n];
    r += v;
    for (int a = 0; a < 3; a++) j[a] += v * CV[q][a];
  }
  *rho = r;
  for (int a = 0; a < 3; a++) u[a] = j[a] / r;
}

/* Even part of the porous equilibrium (Eqs. equilc1, equilc2 without the
 * terms odd in c_q): w_q rho (1 + 4.5 (c_q.u)^2 / eps - 1.5 u.u / eps). */
static void feq_even(double rho, const double *u, double eps, double *out)
{
  double uu = dot3(u, u);
  for (int q = 0; q < Q; q++) {
    double cu = cdot(q, u);
    out[q] = WT[q] * rho * (1.0 + 4.5 * cu * cu / eps - 1.5 * uu / eps);
  }
}

/* Flowchart step f for the fluid lattice at one cell. Free surface (Eq.
 * equilempty): a population that would come from an empty cell is rebuilt as
 * f_q = f^eq_q + f^eq_qbar - f~_qbar(x) with the gas density 1 and the cell's
 * own V' (reading: hydrodynamic equilibrium, V' recovered from the cell's
 * post-collision populations). */
static void stream_fluid(orc *o, int64_t n)
{
  int x, y, z;
  int64_t N = o->N;
  cell_coords(o, n, &x, &y, &z);
  int have_gas_eq = 0;
  double ge[Q];
  for (int q = 0; q < Q; q++) {
    int face = -1;
    int64_t s = pull_source(o, o->p.bc, x, y, z, q, &face);
    double v;
    if (s == ORC_SRC_BOUNCE) {
      v = o->f[(int64_t)OPP[q] * N + n];
    } else if (s == ORC_SRC_PRESSURE) {
      /* anti-bounce-back on the even part of the porous equilibrium at the
       * face density rho_b = 3 eps P_b (P = rho c_s^2 / eps, Section 2), with
       * the velocity of the cell's own post-collision populations */
      double r, u[3], fe[Q];
      post_collision_moments(o, n, &r, u);
      double rb = 3.0 * o->eps[n] * o->p.face_P[face / 2][face % 2];
      feq_even(rb, u, o->eps[n], fe);
      v = -o->f[(int64_t)OPP[q] * N + n] + 2.0 * fe[q];
    } else if (s == ORC_SRC_VELOCITY) {
      /* bounce-back from a face moving with u_b: f_q = f~_qbar + 6 w_q rho
       * (c_q . u_b), rho the cell's own post-collision density */
      double r, u[3];
      post_collision_moments(o, n, &r, u);
      const double *ub = o->p.face_u[face / 2][face % 2];
      v = o->f[(int64_t)OPP[q] * N + n] + 6.0 * WT[q] * r * cdot(q, ub);
    } else if (o->p.free_surface && o->type[s] == ORC_EMPTY) {
      if (!have_gas_eq) {
        double r, u[3];
        post_collision_velocity(o, o->f, n, &r, u);
        feq_hydro(1.0, u, o->eps[n], ge);
        have_gas_eq = 1;
      }
      v = ge[q] + ge[OPP[q]] - o->f[(int64_t)OPP[q] * N + n];
    } else {
      v = o->f[(int64_t)q * N + s];
    }
    o->fs[(int64_t)q * N + n] = v;
  }
}

/* Flowchart step f for the solute lattice (Eq. boltzeqD). Reading of the
 * inlet/outlet faces: a population entering through an INLET face is the
 * equilibrium h^eq_q(eps(x), C_in, V + D grad(eps)/eps) of the receiving cell,
 * with V the cell's streamed bare velocity (V' itself needs the viscosity,
 * which depends on the concentration being formed); a population entering
 * through an OUTLET face is the cell's own post-collision value in the same
 * direction (zero-gradient outflow). Solute flux through the faces is
 * recorded per cell: in = injected - leaving through the inlet, out = leaving
 * through the outlet - re-entered. */
static void stream_solute(orc *o, int64_t n)
{
  int x, y, z;
  int64_t N = o->N;
  cell_coords(o, n, &x, &y, &z);
  double r = 0, j[3] = {0, 0, 0};
  for (int q = 0; q < Q; q++) {
    double v = o->fs[(int64_t)q * N + n];
    r += v;
    for (int a = 0; a < 3; a++) j[a] += v * CV[q][a];
  }
  for (int sp = 0; sp < o->S; sp++) {
    const double *h = o->h + (int64_t)sp * Q * N;
    double *hs = o->hs + (int64_t)sp * Q * N;
    double D = diffusivity_of(o, sp), Cin = C_in_of(o, sp);
    double Vin[3];
    for (int a = 0; a < 3; a++) Vin[a] = j[a] / r + D * o->geps[3 * n + a];
    double fin = 0.0, fout = 0.0;
    for (int q = 0; q < Q; q++) {
      int64_t s = pull_source(o, o->p.sbc, x, y, z, q, NULL);
      double v;
      if (s == ORC_SRC_BOUNCE) {
        v = h[(int64_t)OPP[q] * N + n];
      } else if (s == ORC_SRC_INLET) {
        v = WT[q] * o->eps[n] * Cin * (1.0 + 3.0 * cdot(q, Vin));
        fin += v - h[(int64_t)OPP[q] * N + n];
      } else if (s == ORC_SRC_OUTLET) {
        v = h[(int64_t)q * N + n];
        fout += h[(int64_t)OPP[q] * N + n] - v;
      } else {
        v = h[(int64_t)q * N + s];
      }
      hs[(int64_t)q * N + n] = v;
    }
    o->cell_in[sp * N + n] = fin;
    o->cell_out[sp * N + n] = fout;
  }
}

/* Flowchart step g, Eqs. eq:massmacro, eq:massevol, eq:deltamass. Reading:
 * m(x,t+1) = m(x,t) + sum_q dm_q with dm_q = w (f~_qbar(x+c_q) - f~_q(x)),
 * w = 1 if either cell is liquid, w = (lambda(x)+lambda(x+c_q))/2 between two
 * interface cells, and dm_q = 0 towards empty or solid cells; dm is then
 * antisymmetric and the total liquid mass is conserved. */
static void stream_mass(orc *o, int64_t n)
{
  int x, y, z;
  int64_t N = o->N;
  cell_coords(o, n, &x, &y, &z);
  double m = o->m[n];
  for (int q = 1; q < Q; q++) {
    int64_t b = neighbor(o, o->p.bc, x, y, z, q);
    if (b < 0 || o->solid[b] || o->type[b] == ORC_EMPTY) continue;
    double diff = o->f[(int64_t)OPP[q] * N + b] - o->f[(int64_t)q * N + n];
    double w = 1.0;
    if (o->type[n] == ORC_INTERFACE && o->type[b] == ORC_INTERFACE)
      w = 0.5 * (o->lam[n] + o->lam[b]);
    m += w * diff;
  }
  o->mn[n] = m;
}

/* Flowchart steps h, e, i at one cell: moments (Eqs. macros1, macros),
 * viscosity, colour gradient, velocity correction, BGK collision with forcing
 * (Eq. lbe2 with Omega = -(f - f^eq)/tau; reading: the flowchart's "f - Omega"
 * is taken as Eq. lbe2's "f + Omega"), and the solute collision (Eqs. equild,
 * boltzeqD). Reading: C = sum_q h_q / eps, since sum_q h^eq_q = eps C. */
static void collide(orc *o, int64_t n)
{
  int64_t N = o->N;
  double rho = 0, j[3] = {0, 0, 0};
  for (int q = 0; q < Q; q++) {
    double v = o->fs[(int64_t)q * N + n];
    rho += v;
    for (int a = 0; a < 3; a++) j[a] += v * CV[q][a];
  }
  double V[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  double eps = o->eps[n];
  double Cc = 0.0;
  if (o->p.solute) {
    double s = 0;
    for (int q = 0; q < Q; q++) s += o->hs[(int64_t)q * N + n];
    Cc = s / eps;
  }
  double tau = orc_tau_of(&o->p, Cc, o->t);
  double nu = (tau - 0.5) / 3.0;
  double F[3] = {0, 0, 0};
  if (o->p.A != 0.0) colour_gradient(o, n, F);
  double Vp[3], Fe[3], fe[Q], T[Q];
  orc_velocity_solve(V, eps, nu, o->Kinv ? o->Kinv + 9 * n : NULL, o->p.G, o->p.forchheimer,
                     Vp, Fe);
  orc_feq(rho, Vp, eps, tau, o->p.A, F, fe);
  orc_forcing(rho, tau, eps, Vp, Fe, T);
  for (int q = 0; q < Q; q++) {
    double fq = o->fs[(int64_t)q * N + n];
    o->fn[(int64_t)q * N + n] = fq - (fq - fe[q]) / tau + T[q];
  }
  /* every species relaxes towards its own equilibrium with the shared V'
   * (reading R24: species 0's concentration sets the viscosity) */
  for (int sp = 0; sp < o->S; sp++) {
    const double *hs = o->hs + (int64_t)sp * Q * N;
    double *hn = o->hn + (int64_t)sp * Q * N;
    double Cs = Cc;
    if (sp > 0) {
      double s = 0;
      for (int q = 0; q < Q; q++) s += hs[(int64_t)q * N + n];
      Cs = s / eps;
    }
    double D = diffusivity_of(o, sp), tD = tau_D_of(o, sp), Vs[3], he[Q];
    for (int a = 0; a < 3; a++) Vs[a] = Vp[a] + D * o->geps[3 * n + a];
    orc_heq(eps, Cs, Vs, he);
    for (int q = 0; q < Q; q++) {
      double hq = hs[(int64_t)q * N + n];
      hn[(int64_t)q * N + n] = hq - (hq - he[q]) / tD;
    }
    o->out_C[sp * N + n] = Cs;
  }
  o->out_rho[n] = rho;
  for (int a = 0; a < 3; a++) o->out_u[3 * n + a] = Vp[a];
  o->out_C[n] = Cc;
  o->out_nu[n] = nu;
}

enum { FLAG_NONE = 0, FLAG_FILL = 1, FLAG_EMPTYING = 2 };

static int has_neighbor_flag(const orc *o, int64_t n, int flag)
{
  int x, y, z;
  cell_coords(o, n, &x, &y, &z);
  for (int q = 1; q < Q; q++) {
    int64_t b = neighbor(o, o->p.bc, x, y, z, q);
    if (b >= 0 && !o->solid[b] && o->flag[b] == flag) return 1;
  }
  return 0;
}

/* Flowchart step j (Section 3, last paragraph). Reading: an interface cell
 * fills when lambda > 1 + 1e-3 and empties when lambda < -1e-3; an emptying
 * cell next to a filling one stays interface; empty neighbours of a filled
 * cell become interface with f = f^eq(mean rho, mean V') of their liquid and
 * interface neighbours and no mass; liquid neighbours of an emptied cell
 * become interface; the excess mass (m - rho of a filled cell, m of an
 * emptied cell) is shared equally among the neighbours that are interface
 * cells after the re-typing (kept in the cell when there are none). */
static void convert_cells(orc *o)
{
  int64_t N = o->N;
  const double kappa = 1e-3;
  for (int64_t n = 0; n < N; n++) {
    o->flag[n] = FLAG_NONE;
    if (o->solid[n] || o->type[n] != ORC_INTERFACE) continue;
    if (o->lam[n] > 1.0 + kappa)
      o->flag[n] = FLAG_FILL;
    else if (o->lam[n] < -kappa)
      o->flag[n] = FLAG_EMPTYING;
  }
  for (int64_t n = 0; n < N; n++)
    if (o->flag[n] == FLAG_EMPTYING && has_neighbor_flag(o, n, FLAG_FILL))
      o->ntype[n] = 1; /* mark: cancelled */
    else
      o->ntype[n] = 0;
  for (int64_t n = 0; n < N; n++)
    if (o->ntype[n]) o->flag[n] = FLAG_NONE;

  /* new types; ntype doubles as the new-type array from here on */
  uint8_t *newif = (uint8_t *)zalloc(N);
  for (int64_t n = 0; n < N; n++) {
    uint8_t t = o->type[n];
    if (!o->solid[n]) {
      if (o->flag[n] == FLAG_FILL) t = ORC_LIQUID;
      else if (o->flag[n] == FLAG_EMPTYING) t = ORC_EMPTY;
      else if (o->type[n] == ORC_EMPTY && has_neighbor_flag(o, n, FLAG_FILL)) {
        t = ORC_INTERFACE;
        newif[n] = 1;
      } else if (o->type[n] == ORC_LIQUID && has_neighbor_flag(o, n, FLAG_EMPTYING))
        t = ORC_INTERFACE;
    }
    o->ntype[n] = t;
  }
  /* initialise the new interface cells */
  for (int64_t n = 0; n < N; n++) {
    if (!newif[n]) continue;
    int x, y, z;
    cell_coords(o, n, &x, &y, &z);
    double rs = 0, us[3] = {0, 0, 0};
    int cnt = 0;
    for (int q = 1; q < Q; q++) {
      int64_t b = neighbor(o, o->p.bc, x, y, z, q);
      if (b < 0 || o->solid[b] || newif[b]) continue;
      if (o->ntype[b] != ORC_LIQUID && o->ntype[b] != ORC_INTERFACE) continue;
      double r, u[3];
      post_collision_velocity(o, o->fn, b, &r, u);
      rs += r;
      for (int a = 0; a < 3; a++) us[a] += u[a];
      cnt++;
    }
    double r = rs / cnt, u[3] = {us[0] / cnt, us[1] / cnt, us[2] / cnt}, fe[Q];
    feq_hydro(r, u, o->eps[n], fe);
    for (int q = 0; q < Q; q++) o->fn[(int64_t)q * N + n] = fe[q];
    o->out_rho[n] = r;
    for (int a = 0; a < 3; a++) o->out_u[3 * n + a] = u[a];
    o->out_C[n] = 0.0;
    o->out_nu[n] = (orc_tau_of(&o->p, 0.0, o->t) - 0.5) / 3.0;
  }
  /* excess mass */
  double *share = o->cell_in; /* reuse as scratch: excess per interface neighbour */
  for (int64_t n = 0; n < N; n++) {
    share[n] = 0.0;
    if (o->flag[n] == FLAG_NONE) continue;
    int x, y, z;
    cell_coords(o, n, &x, &y, &z);
    int cnt = 0;
    for (int q = 1; q < Q; q++) {
      int64_t b = neighbor(o, o->p.bc, x, y, z, q);
      if (b >= 0 && !o->solid[b] && o->ntype[b] == ORC_INTERFACE) cnt++;
    }
    if (cnt == 0) continue;
    double excess = (o->flag[n] == FLAG_FILL) ? o->mn[n] - o->out_rho[n] : o->mn[n];
    share[n] = excess / cnt;
    o->mn[n] -= excess;
  }
  for (int64_t n = 0; n < N; n++) {
    if (o->solid[n] || o->ntype[n] != ORC_INTERFACE) continue;
    int x, y, z;
    cell_coords(o, n, &x, &y, &z);
    for (int q = 1; q < Q; q++) {
      int64_t b = neighbor(o, o->p.bc, x, y, z, q);
      if (b >= 0 && !o->solid[b] && o->flag[b] != FLAG_NONE) o->mn[n] += share[b];
    }
  }
  for (int64_t n = 0; n < N; n++) {
    if (o->solid[n]) continue;
    o->type[n] = o->ntype[n];
    if (o->type[n] == ORC_LIQUID)
      o->lam[n] = 1.0;
    else if (o->type[n] == ORC_EMPTY)
      o->lam[n] = 0.0;
    else
      o->lam[n] = o->mn[n] / o->out_rho[n];
    if (o->type[n] == ORC_EMPTY) {
      o->out_rho[n] = o->out_C[n] = o->out_nu[n] = 0.0;
      o->out_u[3 * n] = o->out_u[3 * n + 1] = o->out_u[3 * n + 2] = 0.0;
    }
  }
  free(newif);
}

static void step_once(orc *o)
{
  int64_t N = o->N;
  int64_t n;
  o->t += 1; /* flowchart step d */
#pragma omp parallel for schedule(static)
  for (n = 0; n < N; n++)
    if (active(o, n)) stream_fluid(o, n);
  if (o->p.solute) {
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; n++) {
      for (int sp = 0; sp < o->S; sp++) o->cell_in[sp * N + n] = o->cell_out[sp * N + n] = 0.0;
      if (active(o, n)) stream_solute(o, n);
    }
    for (int sp = 0; sp < o->S; sp++) {
      double fin = 0.0, fout = 0.0;
      for (n = 0; n < N; n++) {
        fin += o->cell_in[sp * N + n];
        fout += o->cell_out[sp * N + n];
      }
      o->flux_in[sp] += fin;
      o->flux_out[sp] += fout;
    }
  }
  if (o->p.free_surface) {
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; n++) {
      if (active(o, n))
        stream_mass(o, n);
      else
        o->mn[n] = o->m[n];
    }
  }
  /* colour-gradient field rhohat: the post-stream density (reading, so that
   * the gradient follows the flowchart order stream -> moments -> gradient),
   * or the liquid mass m(t+1) with a free surface (0 in empty cells) */
  if (o->p.A != 0.0) {
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; n++) {
      if (o->solid[n])
        o->rhohat[n] = o->p.wall_rho;
      else if (o->p.free_surface)
        o->rhohat[n] = (o->type[n] == ORC_EMPTY) ? 0.0 : o->mn[n];
      else {
        double r = 0;
        for (int q = 0; q < Q; q++) r += o->fs[(int64_t)q * N + n];
        o->rhohat[n] = r;
      }
    }
  }
#pragma omp parallel for schedule(static)
  for (n = 0; n < N; n++)
    if (active(o, n)) collide(o, n);
  if (o->p.free_surface) {
    for (n = 0; n < N; n++)
      if (active(o, n)) o->lam[n] = o->mn[n] / o->out_rho[n];
    convert_cells(o);
    double *tm = o->m;
    o->m = o->mn;
    o->mn = tm;
  }
  double *tf = o->f;
  o->f = o->fn;
  o->fn = tf;
  if (o->p.solute) {
    double *th = o->h;
    o->h = o->hn;
    o->hn = th;
  }
}

int orc_step(orc *o, int64_t n)
{
  if (!o || n < 0) return -1;
  for (int64_t i = 0; i < n; i++) step_once(o);
  return 0;
}

int64_t orc_time(const orc *o) { return o ? o->t : -1; }

int orc_set_populations(orc *o, const double *f, const double *h)
{
  if (!o) return -1;
  size_t nq = (size_t)o->N * Q * sizeof(double);
  if (f) memcpy(o->f, f, nq);
  if (h && o->p.solute) memcpy(o->h, h, nq);
  return 0;
}

int orc_get_populations(const orc *o, double *f, double *h)
{
  if (!o) return -1;
  size_t nq = (size_t)o->N * Q * sizeof(double);
  if (f) memcpy(f, o->f, nq);
  if (h && o->p.solute) memcpy(h, o->h, nq);
  return 0;
}

int orc_fields(const orc *o, double *rho, double *u, double *C, double *nu)
{
  if (!o) return -1;
  int64_t N = o->N;
  if (rho) memcpy(rho, o->out_rho, N * sizeof(double));
  if (u) memcpy(u, o->out_u, 3 * N * sizeof(double));
  if (C) memcpy(C, o->out_C, N * sizeof(double));
  if (nu) memcpy(nu, o->out_nu, N * sizeof(double));
  return 0;
}

/* Totals in cell order: fluid mass (sum of populations over non-solid cells,
 * or the liquid mass sum m with a free surface), solute sum_q h_q, and the
 * cumulative inlet and outlet solute fluxes. */
int orc_reduce(const orc *o, double out[4])
{
  if (!o) return -1;
  int64_t N = o->N;
  double mass = 0.0, sol = 0.0;
  for (int64_t n = 0; n < N; n++) {
    if (o->solid[n]) continue;
    if (o->p.free_surface) {
      mass += o->m[n];
      continue;
    }
    for (int q = 0; q < Q; q++) mass += o->f[(int64_t)q * N + n];
    if (o->p.solute)
      for (int q = 0; q < Q; q++) sol += o->h[(int64_t)q * N + n];
  }
  out[0] = mass;
  out[1] = sol;
  out[2] = o->flux_in[0];
  out[3] = o->flux_out[0];
  return 0;
}

int orc_species_state(const orc *o, int32_t s, double *C, double out[3], double *h)
{
  if (!o || s < 0 || s >= o->S) return -1;
  int64_t N = o->N;
  const double *hs = o->h + (int64_t)s * Q * N;
  if (C) memcpy(C, o->out_C + (int64_t)s * N, N * sizeof(double));
  if (h) memcpy(h, hs, (size_t)Q * N * sizeof(double));
  if (out) {
    double sol = 0.0;
    for (int64_t n = 0; n < N; n++) {
      if (o->solid[n]) continue;
      for (int q = 0; q < Q; q++) sol += hs[(int64_t)q * N + n];
    }
    out[0] = sol;
    out[1] = o->flux_in[s];
    out[2] = o->flux_out[s];
  }
  return 0;
}

int orc_neighbors(const orc *o, int32_t lattice, int32_t *src)
{
  if (!o || lattice < 0 || lattice > 1) return -1;
  int64_t N = o->N;
  for (int64_t n = 0; n < N; n++) {
    int x, y, z;
    cell_coords(o, n, &x, &y, &z);
    for (int q = 0; q < Q; q++) {
      int32_t v;
      if (o->solid[n])
        v = ORC_SRC_NOT_UPDATED;
      else
        v = (int32_t)pull_source(o, lattice ? o->p.sbc : o->p.bc, x, y, z, q, NULL);
      src[(int64_t)q * N + n] = v;
    }
  }
  return 0;
}

int orc_free_surface_state(const orc *o, uint8_t *type, double *m)
{
  if (!o) return -1;
  if (type) memcpy(type, o->type, o->N);
  if (m) memcpy(m, o->m, o->N * sizeof(double));
  return 0;
}
