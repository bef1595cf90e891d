/*
 * lb.h - C ABI of the GB300 (sm_103a) lattice-Boltzmann library for flow of
 * mixtures through anisotropic porous media, after Mendoza, Wittel and
 * Herrmann, "Simulation of Flow of Mixtures Through Anisotropic Porous Media
 * using a Lattice Boltzmann Model" (arXiv:0912.4230).
 *
 * One lattice ("context") lives on one GPU. The calls follow the paper's
 * statement of the problem (Section 4): the caller sets the porosity field,
 * the permeability-tensor field, the impermeable cells, the relaxation times
 * and the boundary conditions (lb_create), then the initial density, velocity,
 * concentration and cell types (lb_init), advances the coupled fluid + solute
 * update (lb_step), and reads back density, velocity, concentration and
 * viscosity (lb_fields).
 *
 * Conventions (all calls):
 *  - Cell index n = x + nx*(y + ny*z), x fastest. Per-cell vectors are packed
 *    per cell (u[3*n + a]); per-direction arrays are direction-major
 *    (f[q*N + n]) in the library's D3Q19 order (Section 2.1): q = 0 is the rest
 *    vector and q = 1 + 6p + (i-1) is orientation i = 1..6 in reference plane
 *    p = 0 (x-y), 1 (y-z), 2 (z-x); i = 1..4 are the plane's diagonals
 *    counter-clockwise from (+,+), i = 5, 6 are +/- the plane's first axis.
 *  - Pointer arguments may point to host memory or to device memory of the
 *    context's GPU (unified addressing); input arrays are copied and stay
 *    owned by the caller; output arrays are caller-owned and written in full.
 *  - The library owns every device allocation it makes (through the allocator
 *    set by lb_set_allocator, else cudaMalloc) and releases it in lb_destroy.
 *  - Every call returns LB_OK or a negative LB_E* status; no exception or
 *    abort crosses the ABI; lb_last_error gives a message for the context.
 *  - Calls on one context are not thread-safe; distinct contexts are.
 *  - Work is enqueued on the context's stream (lb_set_stream, default: the
 *    legacy default stream). Calls that return data to the caller
 *    (lb_fields, lb_reduce, lb_get_populations, lb_debug_neighbors,
 *    lb_free_surface_state, lb_sync) synchronise that stream first.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx; /* opaque, library-owned */

enum {
  LB_OK = 0,
  LB_EINVAL = -1,        /* invalid argument or field value */
  LB_ENOMEM = -2,        /* device or host allocation failed */
  LB_ECUDA = -3,         /* a CUDA runtime call failed */
  LB_ENONFINITE = -4,    /* a reduction met a NaN or an infinity */
  LB_ETIMEOUT = -5,      /* a bounded device wait gave up */
  LB_EUNSUPPORTED = -6   /* valid request outside what this build implements */
};

/* Face kinds, per axis and side. The fluid lattice takes PERIODIC, WALL
 * (halfway bounce-back, "impermeability" in Section 4), PRESSURE or VELOCITY
 * (the "pressures, flow rate" of Section 4, which gives no method: a
 * population entering through a PRESSURE face is -f~_qbar(x) + 2 w_q rho_b (1
 * + 4.5 (c_q.u)^2/eps - 1.5 u.u/eps), rho_b = 3 eps(x) face_P (P = rho
 * c_s^2 / eps of Section 2), u the velocity of the cell's own post-collision
 * populations; through a VELOCITY face it is f~_qbar(x) + 6 w_q rho (c_q .
 * face_u), rho the cell's own post-collision density). The solute lattice
 * takes PERIODIC, WALL, INLET (populations entering through the face carry
 * the equilibrium of Eq. equild at concentration C_in) or OUTLET
 * (zero-gradient outflow). Both sides of an axis are periodic or neither.
 * A diagonal leaving through two faces takes the first of WALL, VELOCITY,
 * PRESSURE, INLET, OUTLET, and of two faces of one kind the lower axis. */
enum { LB_BC_PERIODIC = 0, LB_BC_WALL = 1, LB_BC_INLET = 2, LB_BC_OUTLET = 3,
       LB_BC_PRESSURE = 4, LB_BC_VELOCITY = 5 };

/* Population storage (the collision always runs in FP32, or FP64 for
 * LB_STORE_FP64). FP32 and FP64 store f_q - w_q and h_q. FP16DEV and BF16DEV
 * store deviations from the equilibrium weights scaled by the cell's own
 * totals: per cell a reference r_f = rho - 1 (and r_h = sum_q h_q), and per
 * population the 16-bit remainder (f_q - w_q)/w_q - r_f (resp. h_q/w_q - r_h)
 * formed against the stored reference, so density and solute content never
 * pass through the 16-bit mantissa. With the solute lattice the remainders of
 * f_q and h_q (species 0) are stored as one 32-bit pair and the references as
 * one FP16 pair per cell; further species and lattices without solute keep
 * their own rows and FP32 references. */
enum { LB_STORE_FP32 = 0, LB_STORE_FP64 = 1, LB_STORE_FP16DEV = 2, LB_STORE_BF16DEV = 3 };

/* Largest number of solute species (lb_params.species). */
enum { LB_MAX_SPECIES = 8 };

/* Free-surface cell types (Section 3). */
enum { LB_CELL_LIQUID = 0, LB_CELL_INTERFACE = 1, LB_CELL_EMPTY = 2 };

/* Classes returned by lb_debug_neighbors for populations not pulled from a
 * cell. */
enum { LB_SRC_NOT_UPDATED = -1, LB_SRC_BOUNCE = -2, LB_SRC_INLET = -3, LB_SRC_OUTLET = -4,
       LB_SRC_PRESSURE = -6, LB_SRC_VELOCITY = -7 };

typedef struct {
  int32_t nx, ny, nz;   /* lattice size, each >= 1 */
  int32_t bc[3][2];     /* fluid faces [axis x,y,z][low, high] */
  int32_t sbc[3][2];    /* solute faces; must be WALL where bc is WALL */
} lb_domain;

typedef struct {
  double tau;           /* fluid relaxation time (visc_law 0), > 1/2 */
  int32_t visc_law;     /* 0 constant tau; 1 tau = tau0 + (tau1-tau0)*clamp(C,0,1);
                           2 Eq. nuall: nu = nu_g (1 + a e^{alpha t}) e^{beta (1-C)},
                           tau = 3 nu + 1/2, t = step index (0 at lb_init) */
  double tau0, tau1;    /* visc_law 1, each > 1/2 */
  double nu_g, a, alpha, beta; /* visc_law 2 */
  double G[3];          /* body force per unit mass, Eq. forcement */
  double A;             /* surface-tension strength, Eqs. equilc1/equilc2 (0 = off) */
  double wall_rho;      /* colour-gradient density seen at solid cells and
                           wall faces (wetting); used when A != 0 */
  double forchheimer;   /* Forchheimer drag, >= 0 (0 = off). The paper names the
                           term without an equation; this build takes the
                           porous-flow model it builds on: F^ext gains
                           -eps F_eps |V'| K^-1/2 V' with F_eps = forchheimer *
                           1.75 / sqrt(150 eps^3) (Ergun) and the implicit V'
                           of Eq. expandV solved with it. Needs a diagonal K
                           (a full tensor returns LB_EUNSUPPORTED); no effect
                           without K. */
  int32_t solute;       /* 1: solute lattice on (Section 2.2) */
  double tau_D;         /* solute relaxation time, > 1/2; D = (tau_D - 1/2)/3 */
  double C_in;          /* concentration entering through INLET faces */
  int32_t free_surface; /* 1: free-surface cell types and liquid mass (Section 3);
                           requires solute = 0 and no permeability (K6 = NULL) */
  int32_t storage;      /* LB_STORE_* */
  int32_t check_every;  /* every this many steps the step kernel also sums each
                           warp's mass and solute and checks the sums for
                           NaN/Inf (0 = never) */
  int32_t kernel;       /* step kernel: 0 automatic (= 1), 1 one thread per cell
                           with direct loads, 2 row-pipelined with shared-memory
                           staging by bulk asynchronous copies (needs the solute
                           lattice, a permeability field, nx = 128 or 256, FP32
                           storage, no free surface), 3 row-staged: persistent
                           blocks of rows, each thread copying its next cell's
                           inputs to shared memory (cp.async) while it computes
                           the current one (FP32/FP64 storage, no free surface).
                           Kernels 2 and 3 return LB_EUNSUPPORTED where they do
                           not apply (also with PRESSURE or VELOCITY faces). All
                           compute the same arithmetic. */
  double face_P[3][2];      /* pressure of each PRESSURE face [axis][side] */
  double face_u[3][2][3];   /* velocity of each VELOCITY face [axis][side][xyz] */
  int32_t species;          /* solute species, 1..LB_MAX_SPECIES (0 = 1). The paper
                               keeps the solute on its own lattice to allow
                               several species (Section 2.2): each species is a
                               D3Q19 lattice of Eqs. equild/boltzeqD with its own
                               tau_D and inlet concentration, all sharing V';
                               species 0's C sets the viscosity law. Needs
                               solute = 1; with more than one species only the
                               per-cell kernel runs (kernels 2 and 3 return
                               LB_EUNSUPPORTED) and there is no free surface. */
  double species_tau_D[LB_MAX_SPECIES]; /* tau_D of species s >= 1 (species 0: tau_D), > 1/2 */
  double species_C_in[LB_MAX_SPECIES];  /* inlet concentration of species s >= 1 (species 0: C_in) */
} lb_params;

/* Create a lattice (flowchart of Section 4: the porosity field, the
 * permeability fields, the relaxation times and the boundary conditions are
 * set before the distributions are initialised). Sizes: nz <= 65535 and
 * 19 * nx * ny * nz < 2^31 (LB_EUNSUPPORTED beyond).
 *   porosity  N floats, 0 < eps <= 1 in every non-solid cell (Eq. momentum).
 *   K6        N*6 floats per cell (K_xx, K_yy, K_zz, K_xy, K_yz, K_zx), a
 *             symmetric positive-definite permeability tensor (Eq. forcement);
 *             NULL = infinite permeability (no Darcy force). Diagonal tensors
 *             (all off-diagonals zero) use a 3-value inverse per cell.
 *   solid     N bytes, nonzero = impermeable cell (never updated; links into
 *             it bounce back).
 * Returns LB_EINVAL for bad sizes, face kinds, tau <= 1/2, eps out of range or
 * a K that fails a Cholesky test, forchheimer < 0; LB_EUNSUPPORTED for
 * forchheimer != 0 with a non-diagonal K, free_surface together with solute
 * or K6, or PRESSURE/VELOCITY faces together with free_surface or A != 0;
 * LB_ENOMEM/LB_ECUDA on device failures. *out is NULL on failure. */
int lb_create(const lb_domain *domain, const float *porosity, const float *K6,
              const uint8_t *solid, const lb_params *params, lb_ctx **out);

/* Enqueue all further work of the context on this cudaStream_t. With
 * ctx = NULL: the stream on which later lb_create calls of this thread do
 * their own copies and set-up kernels, and the initial stream of the
 * contexts they create (default: the legacy default stream). */
int lb_set_stream(lb_ctx *ctx, void *cuda_stream);

/* Initial fields (flowchart steps a-c, Section 4): f = f^eq (Eqs. equilc1,
 * equilc2) at density rho0 and velocity u0 (taken as V'), h = h^eq (Eq.
 * equild) at concentration C0; t = 0.
 *   rho0 N, u0 3N, C0 N per solute species, species-major (required iff
 *   solute; species s at C0 + s*N), cell_type N (LB_CELL_*,
 *   required iff free_surface), lambda0 N liquid fraction (NULL: 1 liquid,
 *   0.5 interface, 0 empty), f_scale 19*N factors multiplying the initial f
 *   (NULL = 1; seeded perturbations). Solid cells are ignored. rho0, u0, C0
 *   and f_scale in memory the GPU can address (device, managed, pinned host)
 *   are read in place by the initialisation on the context's stream (keep
 *   them until lb_sync); others are copied before lb_init returns. */
int lb_init(lb_ctx *ctx, const float *rho0, const float *u0, const float *C0,
            const uint8_t *cell_type, const float *lambda0, const float *f_scale);

/* Overwrite / read the post-collision populations as absolute FP64 values
 * (19*N each, direction-major; h ignored or untouched without solute). */
int lb_set_populations(lb_ctx *ctx, const double *f, const double *h);
int lb_get_populations(lb_ctx *ctx, double *f, double *h);

/* Advance n time steps (flowchart steps d-j, Section 4): stream f and h with
 * periodic wrap, halfway bounce-back and inlet/outlet faces (Eqs. lbe2,
 * boltzeqD); moments (Eqs. macros1, macros); viscosity from the law; colour
 * gradient (Eq. macros) when A != 0; V' and the Darcy force (Eqs. forcement,
 * expandV); BGK collision with forcing (Eqs. coeffforce1, equilc1, equilc2)
 * and the solute collision (Eq. equild); with a free surface also the mass
 * exchange, empty-neighbour reconstruction and cell re-typing (Section 3).
 * Enqueued asynchronously; launch errors return LB_ECUDA. */
int lb_step(lb_ctx *ctx, int64_t n);

/* CUDA graphs for lb_step and lb_step_batch (no counterpart in the paper;
 * default on). While a lattice's launches repeat exactly from one step pair
 * to the next (no time-dependent viscosity law, check_every 0 or 1; the free
 * surface keeps its tile lists and stamps on the device, so it qualifies),
 * the calls capture two steps, one of each buffer parity, into a
 * graph once and replay it for all but the last step of the call, which is
 * launched directly and exports the fields; the steps compute exactly what
 * direct launches compute. A batch graph is kept by the batch's first
 * context for its members in that order and parity. enable = 0 drops the
 * context's graphs and launches every step directly. Synchronises the
 * context's stream. */
int lb_set_graphs(lb_ctx *ctx, int32_t enable);

/* Test hook: bit 0 set when the context holds a captured lb_step graph, bit 1
 * when it holds a batch graph (as the first context of a batch). */
int lb_debug_graphs(const lb_ctx *ctx);

/* Pick the step kernel and its launch shape by timing (no counterpart in the
 * paper): the per-cell kernel with rows of 32, 64 or 128 threads per block,
 * the row-staged kernel with rows of 32, 64 or 128 threads (FP32/FP64
 * storage), and the row-pipelined kernel where the lattice allows it. Each
 * candidate runs reps side-effect-free launches (input buffer to output
 * buffer without swapping, no flux accumulation, no checks, no field export),
 * so the state and t are unchanged. The fastest is kept for later lb_step
 * calls. *choice (may be NULL) receives the row width for the per-cell
 * kernel, 1000 + the row width for the row-staged kernel, 256 for the
 * row-pipelined kernel, or 0 when nothing was tuned (free surface or surface
 * tension keep fixed launches). Results of a step do not depend on the choice
 * beyond the order of the FP64 flux sums. */
int lb_autotune(lb_ctx *ctx, int32_t reps, int32_t *choice);

/* Advance several lattices by the same n steps (continuous batching; no
 * counterpart in the paper). Per step, a lattice whose per-cell launch alone
 * fills the GPU (at least 6 blocks per SM), or that has pressure or velocity
 * faces, takes that launch; the smaller
 * lattices share one persistent launch per 64 lattices over a work list of
 * their cell blocks, their arguments travelling in the launch's parameters.
 * Each lattice computes exactly what lb_step(n) with the per-cell kernel
 * computes.
 * All contexts: same storage, same permeability mode (none / diagonal / full),
 * same solute setting, no free surface, A = 0 (LB_EUNSUPPORTED otherwise).
 * Work is enqueued on the first context's stream; the contexts' own streams
 * are not used. */
int lb_step_batch(lb_ctx *const *ctxs, int32_t n, int64_t steps);

/* Macroscopic fields after the last step (or lb_init): rho, u = V' (3 per
 * cell), C and the kinematic viscosity nu = (tau - 1/2)/3. Any pointer may be
 * NULL. Solid and empty cells read 0. Returns LB_ENONFINITE if a reduction of
 * a previous step flagged NaN/Inf. */
int lb_fields(lb_ctx *ctx, float *rho, float *u, float *C, float *nu);

/* FP64 totals of the current state, summed in a fixed order: fluid mass
 * (sum of populations over non-solid cells; with a free surface the liquid
 * mass sum m, Eq. eq:massmacro), solute sum_q h_q, and the cumulative solute
 * fluxes through INLET and OUTLET faces since lb_init (in: entered minus
 * left through inlets; out: left minus re-entered through outlets). Any
 * pointer may be NULL. */
int lb_reduce(lb_ctx *ctx, double *mass, double *solute, double *flux_in,
              double *flux_out);

/* Test hook: for lattice 0 (fluid) or 1 (solute), src[q*N + n] = the cell the
 * population q of cell n is pulled from, or an LB_SRC_* class. */
int lb_debug_neighbors(lb_ctx *ctx, int32_t lattice, int32_t *src);

/* Test hook for failure detection (no counterpart in the paper): one warp
 * waits, with the bounded wait of the step kernels' barrier waits, on a
 * shared-memory barrier that nothing completes. The wait gives up after
 * limit_ns (0 < limit_ns <= 2e9), sets the context's timeout status and the
 * call returns LB_ETIMEOUT, as a step whose wait gave up would at the next
 * check. The context stays usable; the status is cleared by lb_init. */
int lb_debug_wait_timeout(lb_ctx *ctx, int64_t limit_ns);

/* Solute species s (0 <= s < species): its concentration field as exported
 * by the last step of the latest lb_step call (C, N floats), its totals
 * {sum_q h_q over non-solid cells, cumulative inlet flux, cumulative outlet
 * flux} (totals, 3 doubles; the fluxes as in lb_reduce) and its populations h_q
 * (h, 19 N doubles, as lb_get_populations). Any pointer may be NULL; host or
 * device pointers. LB_EINVAL for s out of range or without solute. */
int lb_species_state(lb_ctx *ctx, int32_t s, float *C, double *totals, double *h);

/* Free-surface state: cell types (LB_CELL_*) and liquid mass m per cell
 * (in the collision precision, widened to double). */
int lb_free_surface_state(lb_ctx *ctx, uint8_t *type, double *mass);

/* Wait for the context's stream; reports LB_ENONFINITE like lb_fields. */
int lb_sync(lb_ctx *ctx);

/* Steps taken since lb_init. */
int64_t lb_time(const lb_ctx *ctx);

/* Message of the context's last failure ("" if none); for a NULL context the
 * message of the last failed call without a context on this thread
 * (lb_create, lb_bytes_required, lb_totals_noalloc). */
const char *lb_last_error(const lb_ctx *ctx);

/* Release the context and all its device memory (NULL is a no-op). */
void lb_destroy(lb_ctx *ctx);

/* Device memory one lattice takes (no counterpart in the paper; it serves
 * admission by an HBM budget): the bytes lb_create, lb_init and the stepping,
 * export and totals calls (lb_step, lb_step_batch, lb_fields, lb_reduce)
 * allocate for a lattice of this domain and these parameters, each block
 * counted in 256-byte granules as the packed arena hands them out, with the
 * larger of the creation and initialisation staging blocks (the first is
 * released before the second is taken) and the lattice's share of a batch
 * work list (8 bytes per block of its per-cell launch, held by the first
 * context of an lb_step_batch call). Computed from the same layout that
 * lb_create allocates by; host arithmetic only, no device is touched.
 *   k_rows   rows of K^-1 kept: 0 (K NULL), 3 (a diagonal tensor field) or
 *            6 (a full tensor field; also the bound when unknown);
 *   f_scale  nonzero if lb_init will be given f_scale.
 * Population exchange calls (lb_get_populations, lb_set_populations,
 * lb_species_state with h, lb_debug_neighbors, lb_free_surface_state with
 * mass) stage up to 19 N doubles more. Returns LB_OK or LB_EINVAL. */
int lb_bytes_required(const lb_domain *dom, const lb_params *prm, int32_t k_rows,
                      int32_t f_scale, size_t *bytes);

/* Route the library's device allocations through caller functions (for
 * example a framework's caching allocator); both NULL restores cudaMalloc.
 * Affects contexts created afterwards (process-wide; safe to call while other
 * threads create contexts: each takes the hooks in force when it starts).
 * alloc returns NULL on failure; release must accept every pointer alloc
 * returned, and a context keeps the hooks it was created with. */
int lb_set_allocator(void *(*alloc)(size_t bytes, void *user),
                     void (*release)(void *ptr, void *user), void *user);

/* Allocation-free totals (the paper has no counterpart; this serves callers
 * that cannot allocate device memory where they need the totals, e.g. code
 * whose device memory is all reserved up front by a framework's pool, or a
 * loop that must not pay the device-wide synchronisation of cudaMalloc and
 * cudaFree). Computes the FP64 mass and solute totals of lb_reduce (every
 * stored value widened to FP64 here; lb_reduce sums a cell's 19 values in
 * FP32 first, which differs by at most 18 * 2^-24 * sum_q |f_q - w_q| per
 * cell), but of caller-owned device arrays and with no device allocation:
 *   f        19*n_cells floats in device memory, the FP32 storage form
 *            f_q - w_q, direction-major (f[q*n_cells + n]);
 *   h        19*n_cells floats h_q in device memory, or NULL (solute 0);
 *   solid    n_cells bytes in device memory, nonzero = skipped, or NULL;
 *   out      2 doubles (mass, solute), host or device memory;
 *   stream   cudaStream_t the work is enqueued on; the call waits for it.
 * The per-block partial sums live in one fixed array of the library image,
 * (2 * 65536 + 2) doubles on every GPU that loads the library, held until
 * the process exits; so n_cells must be <= 16777216 (LB_EINVAL beyond).
 * The first call on each device looks up that array's device address (a
 * runtime call) and keeps it for the life of the process, so make that first
 * call before any stream capture; a cudaDeviceReset of a device the call has
 * been used on is not supported afterwards (the kept address would be
 * stale). Every call ends by waiting for `stream` (the totals are in `out`
 * when it returns). All calls on a device share the array: calls that
 * overlap on the GPU race. Returns LB_OK, LB_EINVAL or LB_ECUDA; the message
 * of a failure is lb_last_error(NULL) on the calling thread. */
int lb_totals_noalloc(const float *f, const float *h, const uint8_t *solid, int64_t n_cells,
                      double *out, void *stream);

/* Packed lattice arena (no counterpart in the paper): one region of device
 * memory from which the lattices of a serving loop are sub-allocated, so
 * that admission by an HBM budget is admission into one fixed region.
 * First-fit over an address-ordered free list, blocks aligned to 256 bytes,
 * neighbouring free blocks merged on release; thread-safe.
 *   lb_arena_create  base: a region of `bytes` device memory owned by the
 *                    caller (for example one framework tensor), or NULL: the
 *                    arena allocates it with cudaMalloc and frees it in
 *                    lb_arena_destroy. *out is NULL on failure.
 *   lb_arena_use     route the device allocations of contexts created
 *                    afterwards into the arena (as lb_set_allocator does);
 *                    NULL restores cudaMalloc. An arena must outlive the
 *                    contexts allocated from it.
 *   lb_arena_alloc / lb_arena_free  one block (NULL when nothing fits); a
 *                    pointer that is not the start of a live block of the
 *                    arena (NULL, outside the region) is ignored.
 *   lb_arena_stats   bytes in use, the largest free block, the peak use and
 *                    the number of live blocks (any pointer may be NULL).
 * The bookkeeping never touches the region, so a host region serves for
 * tests of the allocator. */
typedef struct lb_arena lb_arena;
int lb_arena_create(void *base, size_t bytes, lb_arena **out);
void lb_arena_destroy(lb_arena *arena);
int lb_arena_use(lb_arena *arena);
void *lb_arena_alloc(lb_arena *arena, size_t bytes);
void lb_arena_free(lb_arena *arena, void *ptr);
int lb_arena_stats(const lb_arena *arena, size_t *used, size_t *largest_free, size_t *peak,
                   size_t *blocks);

#ifdef __cplusplus
}
#endif
#endif /* LB_H */
