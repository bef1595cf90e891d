/*
 * Oracle for the porous-media lattice-Boltzmann scheme of Mendoza, Wittel and
 * Herrmann, "Simulation of Flow of Mixtures Through Anisotropic Porous Media
 * using a Lattice Boltzmann Model" (arXiv:0912.4230).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, FP64, cell-by-cell CPU
 * restatement of the scheme, written so that each step can be checked against
 * the paper by eye. Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it. It shares no code, header, table or constant
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Conventions: cell index n = x + nx*(y + ny*z); populations are stored
 * direction-major, pop[q*N + n]; all arrays are caller-owned and copied.
 * With several solute species, per-species arrays follow one another
 * (species-major): C0[s*N + n]; orc_init's C0 holds all species.
 */
#ifndef LB_ORACLE_H
#define LB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_INLET = 2, ORC_OUTLET = 3,
       ORC_PRESSURE = 4, ORC_VELOCITY = 5 };
enum { ORC_LIQUID = 0, ORC_INTERFACE = 1, ORC_EMPTY = 2 };
enum { ORC_MAX_SPECIES = 8 };
/* classes reported by orc_neighbors for populations that do not come from a cell */
enum { ORC_SRC_NOT_UPDATED = -1, ORC_SRC_BOUNCE = -2, ORC_SRC_INLET = -3,
       ORC_SRC_OUTLET = -4, ORC_SRC_EMPTY = -5, ORC_SRC_PRESSURE = -6,
       ORC_SRC_VELOCITY = -7 };

typedef struct {
  int32_t nx, ny, nz;
  int32_t bc[3][2];   /* fluid lattice, [axis][low/high side]: PERIODIC, WALL,
                         PRESSURE or VELOCITY */
  int32_t sbc[3][2];  /* solute lattice: PERIODIC, WALL, INLET or OUTLET */
  double tau;         /* relaxation time for visc_law 0 */
  int32_t visc_law;   /* 0 constant tau, 1 tau linear in C, 2 Eq. nuall */
  double tau0, tau1;  /* visc_law 1: tau = tau0 + (tau1-tau0)*clamp(C,0,1) */
  double nu_g, a, alpha, beta; /* visc_law 2 */
  double G[3];        /* body force (acceleration) */
  double A;           /* surface-tension strength, 0 = off */
  double wall_rho;    /* colour-gradient mass of solid cells (wetting) */
  int32_t solute;     /* 1 = solute lattice on */
  double tau_D;       /* solute relaxation time */
  double C_in;        /* concentration injected at INLET faces */
  int32_t free_surface;
  int32_t threads;    /* OpenMP threads, <= 0 = library default */
  double forchheimer; /* multiplier c_F of the Ergun coefficient F_eps (0 = no
                         Forchheimer drag); needs a diagonal or no K */
  double face_P[3][2];      /* pressure of each PRESSURE face */
  double face_u[3][2][3];   /* velocity of each VELOCITY face */
  int32_t species;          /* solute lattices (species), 1..ORC_MAX_SPECIES; 0 = 1 */
  double species_tau_D[8];  /* relaxation time of species s >= 1 (species 0: tau_D) */
  double species_C_in[8];   /* inlet concentration of species s >= 1 (species 0: C_in) */
} orc_params;

typedef struct orc orc;

orc *orc_create(const orc_params *p, const double *eps, const double *K6,
                const uint8_t *solid);
int orc_init(orc *o, const double *rho0, const double *u0, const double *C0,
             const uint8_t *type, const double *lambda0, const double *f_scale);
int orc_set_populations(orc *o, const double *f, const double *h);
int orc_get_populations(const orc *o, double *f, double *h);
int orc_step(orc *o, int64_t n);
int orc_fields(const orc *o, double *rho, double *u, double *C, double *nu);
int orc_reduce(const orc *o, double out[4]);
/* Species s (0 <= s < species): its concentration field C (may be NULL), its
 * totals out = {sum_q h_q, cumulative inlet flux, outlet flux} (may be NULL)
 * and its populations h (19 N, may be NULL). */
int orc_species_state(const orc *o, int32_t s, double *C, double out[3], double *h);
int orc_neighbors(const orc *o, int32_t lattice, int32_t *src);
int orc_free_surface_state(const orc *o, uint8_t *type, double *m);
int64_t orc_time(const orc *o);
void orc_destroy(orc *o);

/* Single-cell pieces, exposed so that tests can pin them one by one. */
void orc_velocity_set(int32_t *c, double *w, int32_t *opp);
void orc_feq(double rho, const double *u, double eps, double tau, double A,
             const double *F, double *out);
void orc_forcing(double rho, double tau, double eps, const double *u,
                 const double *Fext, double *out);
void orc_velocity_solve(const double *V, double eps, double nu,
                        const double *Kinv9, const double *G, double cF,
                        double *Vp, double *Fext);
void orc_heq(double eps, double C, const double *Vstar, double *out);
double orc_tau_of(const orc_params *p, double C, int64_t t);

#ifdef __cplusplus
}
#endif
#endif
