/*
 * lbmtree.h -- C ABI of the B300 collide-and-stream library for cell-centred, non-uniform
 * (quadtree/octree) lattice Boltzmann grids.
 *
 * The calls follow the statement of the problem in Coreixas & Latt, arXiv 2504.04465:
 * build the tree and its neighbour lists on the host (Secs. 4.3-4.4), choose the lattice and
 * collision model (Appendix A), set the boundaries (Appendix A.3), advance the levels with the
 * asynchronous schedule of Sec. 4.5 and the Rohde coalescence/explosion of Sec. 3.2, and read
 * the macroscopic fields.
 *
 * Conventions
 *   - Every function returns an int status: LBM_OK (0) or a negative LBM_ERR_* code.  The
 *     message of the last failure on the calling thread is returned by lbm_last_error(); the
 *     string is owned by the library and valid until the next call on that thread.
 *   - No C++ exception crosses the ABI.  Device code never traps: kernels that detect a problem
 *     (non-converged Newton solve) record it in a device status word that lbm_sync() returns.
 *   - The library owns every device array.  Host input arrays are copied during the call and may
 *     be freed afterwards.  Host views returned by the library stay valid until lbm_destroy().
 *   - All device work is issued on the stream given to lbm_create() (NULL = a non-blocking
 *     stream created and owned by the context).  lbm_step() is asynchronous; calls that return host data synchronise the stream.
 *   - Levels: level 0 is the finest; a level-i cell has edge 2^i in finest units.  Coordinates
 *     are integer cell indices at the cell's own level.
 */
#ifndef LBMTREE_H
#define LBMTREE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define LBM_OK               0
#define LBM_ERR_ARG         -1   /* invalid argument (null pointer, out-of-range enum)        */
#define LBM_ERR_STATE       -2   /* call out of order (e.g. step before build/init)           */
#define LBM_ERR_CUDA        -3   /* a CUDA runtime call failed                                 */
#define LBM_ERR_OOM         -4   /* device or host allocation failed                           */
#define LBM_ERR_GRID        -5   /* the requested grid violates a builder invariant            */
#define LBM_ERR_NEWTON      -6   /* a Newton solve did not converge (result still written)     */
#define LBM_ERR_NONFINITE   -7   /* a NaN/Inf was found by a reduction (lbm_conserved)         */
#define LBM_ERR_UNSUPPORTED -10  /* combination of lattice/model/storage not built            */

/* ---------------------------------------------------------------- enums */
/* Velocity sets of Appendix A, Tab. lattices_structure (D3Q27: tensor product of D1Q3). */
#define LBM_D2Q9   9
#define LBM_D2Q13 13
#define LBM_D2Q21 21
#define LBM_D2Q37 37
#define LBM_D3Q27 27

/* Collision models (Appendix A): BGK and recursive regularization with the Hermite equilibrium
 * of Eq. GenEq (weakly compressible: D2Q9 and D3Q27 on their tensor-product bases, all storage
 * formats; D2Q13 and D2Q21 on every component up to order 3, FP64 and FP32); compressible
 * polyatomic DDF (Eqs. gEq, polyTemp) with the thermal polynomial equilibrium (D2Q37) or with the
 * numerical max-entropy equilibrium of Eq. exponential solved by Newton-Raphson in FP64 or FP32
 * (D2Q13, D2Q21 and D2Q37, Appendix A.2; on D2Q13 the FP32 solve with FP32 populations only). */
#define LBM_BGK             1
#define LBM_RR              2
#define LBM_COMP_POLY       3
#define LBM_COMP_NUMERICAL  4
/* Two-relaxation-time collision (D2Q9, D3Q27; F64 and F32 storage): the parts of f - f_eq even
 * and odd under xi -> -xi relax with 1/tau (tau from nu0, the shear viscosity) and with the rate
 * fixed by Lambda = (tau - 1/2)(tau_odd - 1/2) (trt_magic below); needs nu0 > 0. */
#define LBM_TRT             5

/* Population storage.  F64/F32: plain values.  F16DEV: binary16 deviations
 * delta_i = f_i/(w_i rho_ref) - 1 (and for g: g_i/(w_i rho_ref (2Cv-D) T0) - 1), arithmetic in
 * FP32.  The Newton solve and the conservation reductions are FP64 in every storage mode. */
#define LBM_F64     1
#define LBM_F32     2
#define LBM_F16DEV  3

/* Boundary kinds for the six faces (Appendix A.3), applied on `reach` layers.  PERIODIC wraps.
 * EQ_DIRICHLET imposes rho, u, T through the equilibrium; EQ_DIRICHLET_RHO imposes u, T and
 * extrapolates rho from the nearest interior cell along the face normal; NEUMANN copies every
 * population of that interior cell.  WALL: halfway bounce-back at the face plane (no boundary
 * layer): a link whose source leaves the domain through wall faces only returns the cell's own
 * opposite post-collision population plus Ladd's moving-wall term 2 w_i rho_w (xi_i . u_w)/c_s^2
 * (rho_u_T = {rho_w, u_w}; a link leaving through several wall faces at once takes the mean of
 * their rho_w u_w; moving walls with the weakly compressible models only).  No ghost layer may
 * lie within the lattice reach of a wall face (LBM_ERR_GRID).
 * Faces: 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+. */
#define LBM_PERIODIC          0
#define LBM_EQ_DIRICHLET      1
#define LBM_EQ_DIRICHLET_RHO  2
#define LBM_NEUMANN           3
#define LBM_WALL              4

/* Initial guess of the Newton solve.  WARM: the multipliers stored in the cell (carried through
 * coalescence/explosion, Sec. 3.2).  ZERO: lambda = 0.  POLY: weighted least-squares fit of
 * -1 - ln f_poly (f_poly the thermal Hermite equilibrium, positive populations only).
 * MLP: a small network (below) trained on equilibria the solver produces; Newton still runs to
 * the same tolerance, so the result does not depend on the guess beyond the tolerance. */
#define LBM_GUESS_WARM  0
#define LBM_GUESS_ZERO  1
#define LBM_GUESS_POLY  2
#define LBM_GUESS_MLP   3   /* the context's network (lbm_mlp_set) */

/* Analytic solids (cells whose centre lies inside are solid, level 0 only). */
#define LBM_SOLID_SPHERE 1   /* p = {cx, cy, cz, radius}                (finest units)      */
#define LBM_SOLID_NACA   2   /* p = {chord, x_le, y_axis, thickness}    symmetric 4-digit,
                                closed trailing edge, zero angle of attack (2D)          */

/* Cell types reported by lbm_cells(). */
#define LBM_CELL_FLUID   1
#define LBM_CELL_CGHOST  2   /* coarse ghost: collides, coalesced from / exploded to children */
#define LBM_CELL_FGHOST  3   /* fine ghost: streams only                                       */
#define LBM_CELL_BC      4   /* boundary layer cell                                            */
#define LBM_CELL_SOLID   5

typedef struct lbm_ctx lbm_ctx;

typedef struct {
    double nu0;          /* kinematic viscosity in level-0 lattice units (0 = inviscid)        */
    double T0;           /* reference temperature (compressible); 0 = lattice c_s^2             */
    double gamma;        /* specific heat ratio of the DDF (Cv = 1/(gamma-1))                   */
    int    sensor_on;    /* kinetic shock sensor, Eqs. DeltaAvg / shock_function                */
    double sensor_A;     /* value of alpha on [0.1, 1)                                          */
    double newton_tol;   /* stop when max |G| < tol; <= 0: 1e-12 (FP64) or 1e-5 (FP32 solve)      */
    int    newton_max_iter;
    int    guess;        /* LBM_GUESS_*                                                         */
    double rho_ref;      /* reference density of the F16DEV storage (1.0)                       */
    int    newton_fp32;  /* 1: Newton of the numerical equilibrium in FP32 arithmetic (the
                            paper's single-precision threshold is 1e-5); multipliers kept in
                            FP64 between steps.  0 (default): FP64 Newton.                     */
    int    trace_eq;     /* LBM_RR on D2Q9/D3Q27 (F64, F32 storage): equilibrate the trace of the
                            second-order moments (Appendix A, after Eq. a1Rec; bulk relaxation
                            time one): Pi is replaced by its deviatoric part in the recursion  */
    double trt_magic;    /* LBM_TRT: Lambda = (tau - 1/2)(tau_odd - 1/2); <= 0: 1/4            */
} lbm_collision_params;

typedef struct { int level; int64_t lo[3]; int64_t hi[3]; } lbm_box;     /* finest units */
typedef struct { int kind; double p[8]; } lbm_shape;

typedef struct {
    int64_t n_cells[8];          /* allocated non-absent cells per level                      */
    int64_t n_blocks[8];
    double  n_eq;                /* sum_i n_i / 2^i over non-solid cells (Sec. 7.5)            */
    int     n_levels;
    int     block[3];            /* cell block shape                                          */
    int64_t newton_iter_sum;     /* Newton iterations summed over all collisions              */
    int64_t newton_updates;      /* collisions that ran a Newton solve                        */
    int64_t newton_nonconverged;
    int64_t newton_hist[16];     /* histogram of iterations per collision (last bin: >= 15)   */
    int64_t fine_iterations;     /* fine iterations advanced since initialisation             */
    int64_t kernel_launches;     /* step-kernel launches issued since initialisation          */
    int64_t device_bytes;        /* device memory held by the context                         */
    int64_t cell_updates;        /* cell updates per coarse step (sum_i n_i 2^(L-1-i))          */
    int64_t n_general_blocks[8]; /* blocks with ghost, boundary or solid-adjacent cells         */
} lbm_stats_t;

/* ---------------------------------------------------------------- lifecycle */
/* Create a context bound to `device` and `stream` (cudaStream_t, or NULL for a stream owned by
 * the context).  dim = 2 or 3.
 * device < 0 makes a host-only context: grids can be built and inspected, nothing runs. */
/* Velocity count, dimension, reach and lattice temperature c_s^2 of a velocity set (LBM_D2Q*,
 * LBM_D3Q27; D2Q37's c_s^2 is the one the library derives from the isotropy conditions). */
int lbm_lattice_info(int lattice, int* Q, int* D, int* reach, double* cs2);
/* Device memory of the grid's arrays (populations, tables, multipliers) from the caller's
 * allocator, for instance a framework's caching allocator: alloc(bytes, user) returns device
 * memory on the context's device, aligned to at least 16 bytes (NULL on failure; a less aligned
 * block is returned to free() and the build fails), free(ptr, user) returns it.  Set before
 * lbm_build_grid; NULL restores cudaMalloc.  Temporary buffers of initialisation, readout and
 * training still use cudaMalloc. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* user;
} lbm_allocator;
int lbm_set_allocator(lbm_ctx* ctx, const lbm_allocator* allocator);
int lbm_create(lbm_ctx** out, int dim, int device, void* stream);
/* Release every device and host resource of the context.  NULL is accepted. */
int lbm_destroy(lbm_ctx* ctx);
const char* lbm_last_error(void);

/* ---------------------------------------------------------------- configuration */
int lbm_set_lattice(lbm_ctx* ctx, int lattice);
int lbm_set_collision(lbm_ctx* ctx, int model, const lbm_collision_params* params);
/* Newton starting point of the numerical equilibrium (LBM_GUESS_*), also on a built and running
 * context (the next step uses it; the captured graph is rebuilt). */
int lbm_set_guess(lbm_ctx* ctx, int guess);
/* Arithmetic (fp32 = 1: FP32, 0: FP64) and tolerance (<= 0: the default of that arithmetic) of
 * the Newton solve, also on a built and running context. */
int lbm_set_newton_precision(lbm_ctx* ctx, int fp32, double tol);
int lbm_set_precision(lbm_ctx* ctx, int storage);
/* Streaming scheme (before lbm_build_grid).  AB (default): two population buffers, pull
 * streaming.  AA: one buffer updated in place (the AA pattern; Sec. 9's outlook): even
 * iterations read and write each cell's own slots (the read reversed), odd iterations gather from
 * the neighbours and write each post-collision population back into the slot its opposite was
 * read from.  Results are bitwise those of AB; population memory is halved.  Single-level grids
 * with periodic, wall and imposed-equilibrium (EQ_DIRICHLET) faces, D2Q9/D3Q27 BGK and RR and
 * D2Q37 polynomial DDF; otherwise lbm_build_grid returns LBM_ERR_UNSUPPORTED. */
#define LBM_STREAM_AB 0
#define LBM_STREAM_AA 1
int lbm_set_streaming(lbm_ctx* ctx, int mode);
/* Far-field relaxation of Eq. relaxation_pressure (weakly compressible models, p = rho c_s^2):
 * before every collision, rho' = rho (1 - sigma) + sigma rho_inf with sigma = 0 for r < r0,
 * sigma_max (r - r0)/(r1 - r0) for r0 <= r < r1 and sigma_max beyond, r the distance of the
 * cell centre from `centre` (finest units; z ignored in 2D); the populations become
 * f + f_eq(rho', u) - f_eq(rho, u) (velocity and non-equilibrium part kept).  sigma_max = 0
 * switches it off (the default).  Errors: LBM_ERR_ARG for r1 <= r0, sigma_max outside [0, 1] or
 * rho_inf <= 0; LBM_ERR_UNSUPPORTED with a compressible model.  Takes effect at the next step. */
int lbm_set_sponge(lbm_ctx* ctx, const double centre[3], double r0, double r1, double sigma_max, double rho_inf);
/* face 0..5; kind LBM_*; rho_u_T = {rho, ux, uy, uz, T} (ignored for PERIODIC/NEUMANN). */
int lbm_set_boundary(lbm_ctx* ctx, int face, int kind, const double rho_u_T[5]);
/* Block shape of the cell layout (x, y, z; z = 1 in 2D).  Defaults 16x16 (2D), 8x4x4 (3D).
 * Each extent must be even and at least the lattice reach.  Must precede lbm_build_grid(). */
int lbm_set_block(lbm_ctx* ctx, int bx, int by, int bz);

/* Compiled variants of the step kernels (occupancy targets): *n variants; minb[k] encodes the
 * resident 128-thread blocks per SM variant k is compiled for as 10 * interior + general
 * (0 = the model's defaults; minb may be NULL, else holds 8 ints).  Codes of 100 and above are the
 * same targets with the interior blocks gathered directly from global memory instead of staged
 * through shared memory (the D3Q27 regularized model in binary16 storage stages by default).  The
 * variants compute the same result; lbm_set_variant() picks one (an autotuner times them).  Both
 * need a built grid. */
int lbm_variants(lbm_ctx* ctx, int* n, int* minb);
int lbm_set_variant(lbm_ctx* ctx, int variant);

/* ---------------------------------------------------------------- grid (Secs. 3.2, 4.3-4.4) */
/* Build the levels, neighbour tables, ghost layers and boundary layers, and allocate the
 * device arrays.  extent: finest-level extent per axis (divisible by 2^(n_levels-1)).
 * boxes: refinement boxes, box.level in [0, n_levels-2]; the region of level i is the union of
 * its boxes (the whole domain for the coarsest level), aligned to 2^(i+1) finest units, each box
 * inside a box of the next coarser level.  solids: analytic shapes at level 0.  Returns
 * LBM_ERR_GRID with a message when an invariant fails (misaligned or non-nested boxes, ghost
 * layers overlapping, a region touching a non-periodic face, a solid closer than the reach to
 * a ghost or boundary layer). */
int lbm_build_grid(lbm_ctx* ctx, const int64_t extent[3], int n_levels,
                   const lbm_box* boxes, int n_boxes, const lbm_shape* solids, int n_solids);
/* The same from a level map instead of boxes (the mesh density field of Sec. 8): level_map holds,
 * for every finest-level cell (x fastest, extent[0] * extent[1] (* extent[2]) bytes, copied),
 * the finest level wanted there, 0 (finest) to n_levels - 1.  The region of level i is every
 * level-(i+1) cell that holds a finest cell wanting level i or finer, so the regions are nested
 * and aligned by construction.  The map must leave room for the ghost layers (about four lattice
 * reaches of level-i cells between the borders of regions i - 1 and i; lbm_amr_level_map
 * grades a map so); otherwise LBM_ERR_GRID as for boxes. */
int lbm_build_grid_map(lbm_ctx* ctx, const int64_t extent[3], int n_levels, const uint8_t* level_map,
                       const lbm_shape* solids, int n_solids);
/* Library-owned host view of the cells (levels ascending, then Morton order of blocks, then
 * x-fastest inside a block).  xyz is n_cells x 3 (z = 0 in 2D).  Valid until lbm_destroy(). */
int lbm_cells(lbm_ctx* ctx, int64_t* n_cells, const int32_t** level, const int32_t** xyz,
              const uint8_t** type);
/* Velocities of the lattice: xi[Q*3] (library-owned), in the population order of the
 * readout calls. */
int lbm_velocities(lbm_ctx* ctx, int* Q, const int32_t** xi);

/* ---------------------------------------------------------------- adaptive mesh refinement (Sec. 8) */
/* Grade a level map in place so that it can be built: for i = 0 .. n_levels - 2, every
 * level-(i+1) cell within 3 reach + 1 level-(i+1) cells (Chebyshev, wrapping where periodic[d])
 * of one holding a finest cell that wants level i or finer gets level i + 1 or finer.  Host only. */
int lbm_grade_level_map(int dim, const int64_t extent[3], int n_levels, int lattice, const int periodic[3],
                        uint8_t* level_map);
/* Level map from the kinetic sensor (Eq. DeltaAvg of the pre-collision state, the criterion of
 * Sec. 8's supersonic airfoil): every finest cell under a bulk or boundary cell whose eps exceeds
 * `threshold` wants level 0; elsewhere fixed_map (NULL: the coarsest level); then graded as
 * above.  level_map: caller-owned, one byte per finest cell, x fastest.  Synchronises. */
int lbm_amr_level_map(lbm_ctx* ctx, double threshold, const uint8_t* fixed_map, uint8_t* level_map);
/* Rebuild the grid from a level map and carry the state over (Sec. 8): a new cell takes the old
 * conserved state at the same level and place (coarse ghosts with their unknown populations
 * coalesced, a fine ghost standing for its coarse-ghost parent), else the old coarser cell
 * holding it (uniform explosion), else the mean of its children resolved the same way
 * (coalescence); f, g and the multipliers alike.  The new state is pre-collision at a coarse
 * synchronisation instant and the level schedule restarts there.  Needs the context at such an
 * instant (LBM_ERR_STATE), two-buffer streaming (LBM_ERR_UNSUPPORTED) and a map the builder
 * accepts (LBM_ERR_GRID: the context is then left without a grid). */
int lbm_remesh(lbm_ctx* ctx, const uint8_t* level_map);

/* ---------------------------------------------------------------- fields */
/* Initialise every cell at equilibrium (Appendix A.3) from host arrays in lbm_cells() order:
 * rho[n], u[dim*n] (SoA: u[d*n + i]), T[n] (NULL for weakly compressible models).  Resets the
 * iteration counter.  Newton multipliers start from the POLY guess. */
int lbm_init_fields(lbm_ctx* ctx, const double* rho, const double* u, const double* T);

/* ---------------------------------------------------------------- stepping (Sec. 4.5) */
/* Advance n_coarse coarse steps (2^(n_levels-1) fine iterations each).  Asynchronous. */
int lbm_step(lbm_ctx* ctx, int64_t n_coarse);
/* Advance n_fine fine iterations (any count; levels stay on the schedule). */
int lbm_step_fine(lbm_ctx* ctx, int64_t n_fine);
/* Use (1) or stop using (0) a captured CUDA graph of two coarse periods in lbm_step(). */
int lbm_use_graph(lbm_ctx* ctx, int on);
/* Wait for the context's stream; return the first device status (LBM_OK, LBM_ERR_NEWTON). */
int lbm_sync(lbm_ctx* ctx);

/* ---------------------------------------------------------------- outputs */
/* rho[n], u[dim*n], T[n] (T may be NULL) of every cell in lbm_cells() order, computed from the
 * populations a cell would collide at the current fine iteration (its streamed populations,
 * with boundary layers applied; coarse-ghost unknowns are not coalesced).  Synchronises. */
int lbm_read_moments(lbm_ctx* ctx, double* rho, double* u, double* T);
/* which = 0: f, 1: g, 2: lambda.  out[Q*n] (lambda: 8*n), SoA by population, in lbm_cells()
 * order, population order of lbm_velocities().  Same state as lbm_read_moments(). */
int lbm_read_populations(lbm_ctx* ctx, int which, double* out);
/* Conserved totals at a coarse synchronisation instant (iteration multiple of 2^(L-1)):
 * out = {mass, momentum_x, momentum_y, momentum_z, energy}, each the sum over bulk, boundary and
 * coarse-ghost cells (unknowns coalesced) of the cell volume 2^(i D) times sum f, sum xi f and
 * sum (|xi|^2 f + g)/2.  FP64, deterministic (fixed-order two-pass reduction through a
 * library-owned scratch array).  LBM_ERR_STATE off a synchronisation instant. */
int lbm_conserved(lbm_ctx* ctx, double out[5]);
int lbm_stats(lbm_ctx* ctx, lbm_stats_t* out);

/* The same totals as lbm_conserved(), for callers that cannot allocate device memory when they
 * need them (a host framework that owns all device memory through its own pool and forbids raw
 * cudaMalloc, a loop that must not trigger the synchronisation an allocation can cause).  No
 * counterpart in the paper.  The call allocates nothing: d_out is the caller's device buffer of
 * 5 doubles {mass, momentum_x, momentum_y, momentum_z, energy}, written asynchronously on the
 * context's stream (read it after lbm_sync()).  The per-block partial sums go to a fixed device
 * array of the library holding at most 524288 blocks (20 MiB, kept by every GPU that loads the
 * library until the process exits); larger grids are rejected with LBM_ERR_ARG.  The first call on
 * a device looks up that array's address, so make it before any stream capture; the address is
 * kept per device and driver context and looked up again if the device's context was recreated.
 * All calls share the array: calls that overlap on the GPU race.  Unlike lbm_conserved, the call
 * does not check the totals for NaN/Inf (they never reach the host): a caller that needs that
 * check tests d_out after lbm_sync().  LBM_ERR_STATE off a synchronisation instant. */
int lbm_conserved_noalloc(lbm_ctx* ctx, double* d_out);

/* ---------------------------------------------------------------- measurement */
/* Floating-point throughput of a fused multiply-add pipe of `device`, the compute denominator
 * of the roofline of compute-bound step kernels (no counterpart in the paper): kind 0 FP32 FMA,
 * 1 FP64 FMA, 2 packed FP32-pair FMA (fma.rn.f32x2, two FMAs per instruction).  One wave of
 * resident 256-thread blocks runs 8 independent FMA chains per thread for `iters` rounds; the
 * best of 5 timed launches after one warm-up gives *flop_per_s (an FMA counts 2 operations) and
 * *ms.  The result is at whatever SM clock the GPU runs at: sample the clock beside it.
 * Allocates a small output buffer; synchronous.  LBM_ERR_ARG for another kind. */
int lbm_pipe_peak(int device, int kind, int iters, double* flop_per_s, float* ms);

/* ---------------------------------------------------------------- checkpoint / restart */
/* Write the state (populations of both buffers, multipliers, fine iteration counter, device
 * status and Newton counters) to a file; synchronous.  lbm_load restores it into a context
 * configured and built the same way (lattice, model, storage, block shape, grid): the file
 * records a signature of these and is rejected (LBM_ERR_STATE) for another configuration. */
int lbm_save(lbm_ctx* ctx, const char* path);
int lbm_load(lbm_ctx* ctx, const char* path);

/* Time every compiled step variant (occupancy targets, lbm_variants) over n_coarse coarse steps
 * (after one warm-up step each) on the context's stream, select the fastest and return it; the
 * steps advance the state.  ms_per_step (optional) receives one time per variant. */
int lbm_autotune(lbm_ctx* ctx, int n_coarse, int* best_variant, float* ms_per_step);

/* ---------------------------------------------------------------- batched cases */
/* Several independent cases (contexts built and initialised on one device) advanced together:
 * each fine iteration launches, per group of cases sharing lattice, model, storage, block
 * shape and step variant, one kernel over the active simple/streaming blocks of all its cases
 * and one over their general blocks, instead of two launches per case.  Cases keep their own
 * state and schedule (a case with L levels advances level i at its own iterations
 * t % 2^i == 0, Sec. 4.5); results are bitwise those of stepping each case alone.  Supported
 * for D2Q9 and D2Q37 (LBM_ERR_UNSUPPORTED otherwise).  The batch reads each case's settings
 * when it is created: a case reconfigured afterwards needs a new batch.  Stepping a case on
 * its own in between is allowed (the batch rebuilds its tables).  Work goes on `stream` (NULL:
 * a stream the batch owns); each case's stream waits for it after every lbm_batch_step. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(lbm_batch** out, lbm_ctx* const* cases, int n, void* stream);
int lbm_batch_destroy(lbm_batch* batch);
/* Capture the cases' common schedule period (2^L fine iterations, L the largest level count)
 * as one CUDA graph and replay it (1) or launch iteration by iteration (0, the default). */
int lbm_batch_use_graph(lbm_batch* batch, int on);
/* Advance every case by n_fine fine iterations of its own finest level (asynchronous). */
int lbm_batch_step(lbm_batch* batch, int64_t n_fine);
/* Wait for the batch and return the first device status of its cases. */
int lbm_batch_sync(lbm_batch* batch);
/* Number of groups, kernel launches issued so far, schedule period in fine iterations. */
int lbm_batch_info(lbm_batch* batch, int* n_groups, int64_t* launches, int64_t* span);

/* ---------------------------------------------------------------- learned Newton guess */
/* A beyond-the-paper extension of the numerical equilibrium (Appendix A, Eq. exponential): a
 * 3 -> 64 -> 64 -> 8 network with tanh hidden layers maps x = (u_x, u_y, T/T0 - 1) to
 * y, and lambda0 = m + s * y is the Newton starting point.  Parameters: one FP32 vector of
 * lbm_mlp_nparams() values [W1 (64x3), b1 (64), W2 (64x64), b2 (64), W3 (8x64), b3 (8)],
 * row-major; weight matrices are used rounded to bfloat16 (nearest even), arithmetic FP32.
 * The training calls work on caller-owned device buffers and the given stream. */
int lbm_mlp_nparams(void);
/* y[n*8] = network(x[n*3]) (x FP64, y FP32). */
int lbm_mlp_forward(const float* d_params, const double* d_x, int64_t n, float* d_y, void* stream);
/* d_grad[nparams] = gradient of L = 1/(2n) sum ||y - t||^2 over the batch, d_loss[0] = L
 * (both overwritten; t[n*8] FP32 targets in normalised units). */
int lbm_mlp_grad(const float* d_params, const double* d_x, const float* d_t, int64_t n, float* d_grad,
                 float* d_loss, void* stream);
/* The same forward pass and gradient with the 64-wide products (layers 2 and 3 and their
 * gradients) on the BF16 tensor cores (warp-level mma.sync m16n8k16, FP32 accumulation): the
 * operands of those products -- the hidden activations, dL/dy and the layer-2 delta -- are
 * rounded to bfloat16 as the weights are; layer 1, tanh, the biases and dW1 stay FP32.
 * Same arguments and outputs as lbm_mlp_forward / lbm_mlp_grad. */
int lbm_mlp_forward_tc(const float* d_params, const double* d_x, int64_t n, float* d_y, void* stream);
int lbm_mlp_grad_tc(const float* d_params, const double* d_x, const float* d_t, int64_t n, float* d_grad,
                    float* d_loss, void* stream);
/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8) of d_params with moments d_m, d_v;
 * step counts from 1. */
int lbm_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int step, float lr, void* stream);
/* Network used by the context when guess = LBM_GUESS_MLP (host parameters, copied; m, s host). */
int lbm_mlp_set(lbm_ctx* ctx, const float* params, const double m[8], const double s[8]);
/* The context's network: FP32 master parameters (trained, before rounding) and m, s (host
 * buffers of lbm_mlp_nparams(), 8 and 8 values).  LBM_ERR_STATE if no network is set. */
int lbm_mlp_get(lbm_ctx* ctx, float* params, double m[8], double s[8]);

typedef struct {
    int steps;              /* Adam steps */
    int batch;              /* samples per step, drawn with replacement */
    double lr, lr_final;    /* learning rate, decayed linearly from lr to lr_final */
    uint64_t seed;          /* initial weights and minibatches (counter-based hash) */
    float final_loss;       /* out: loss of the trained network over all n samples */
    int tensor_cores;       /* 1: gradients by lbm_mlp_grad_tc (BF16 tensor cores), 0: FP32 cores */
} lbm_mlp_train_params;

/* Train the context's network on n device samples: uT[n*3] = (u_x, u_y, T) and the converged
 * multipliers lambda[n*8] (for instance from lbm_newton_batch); the context's model must be
 * LBM_COMP_NUMERICAL (D2Q21 or D2Q37).  m and s are the per-output
 * mean and standard deviation of lambda; training minimises the loss of lbm_mlp_grad on
 * (lambda - m)/s with the project's kernels; the context then uses the network for
 * LBM_GUESS_MLP.  Allocates temporary device memory; synchronous with the context's stream. */
int lbm_mlp_train(lbm_ctx* ctx, const double* d_uT, const double* d_lambda, int64_t n, lbm_mlp_train_params* p);
/* Batched FP64 equilibrium solve of the context's numerical model (D2Q21 or D2Q37): samples uT[n*3] =
 * (u_x, u_y, T) on the device, guess ZERO, POLY or MLP; writes lambda[n*8] and the Newton
 * iterations per sample (-1 if not converged) on the context's stream. */
int lbm_newton_batch(lbm_ctx* ctx, const double* d_uT, int64_t n, int guess, double* d_lambda, int* d_iters);

#ifdef __cplusplus
}
#endif
#endif /* LBMTREE_H */
