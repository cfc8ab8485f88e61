/*
 * ledds.h -- C ABI of the GB300-native coupled LBM-PSM-DEM time step of LEDDS
 * (arXiv 2512.04997).
 *
 * One simulation object couples a D3Q19 BGK lattice with partially saturated cells
 * (Secs. 2.3-2.4) to a discrete-element model of spheres and ellipsoids (Secs. 2.1-2.2).
 * A simulation with nx = ny = nz = 0 is DEM only. Every stage runs as CUDA kernels
 * compiled for sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *  - Return value: LEDDS_OK (0) or a negative LEDDS_ERR_* code; ledds_strerror() names it.
 *  - Units are lattice units: node spacing 1, fluid time step 1. Nodes sit at integer
 *    coordinates 0..n-1 and own the cell [x-1/2, x+1/2]; walls lie halfway, at -1/2
 *    and n-1/2. A DEM-only simulation uses the box given in ledds_dims.
 *  - Pointers prefixed d_ are device pointers owned by the caller; h_ are host pointers.
 *    "on_device" arguments say which of the two a buffer is.
 *  - All device work is enqueued on the stream given to ledds_create and is asynchronous
 *    unless a function says it synchronises.
 *  - The library allocates no device memory: all state lives in the caller's workspace
 *    (ledds_workspace_size / ledds_create). The caller keeps the workspace alive until
 *    ledds_destroy.
 *  - Field arrays are [component][cell] with cell = x + nx*(y + ny*z). Particle state
 *    arrays are [component][particle] ("SoA"); see ledds_read_particles.
 *  - Population order (D3Q19): rest; +x,-x,+y,-y,+z,-z; then (1,1,0),(-1,-1,0),
 *    (1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),
 *    (0,-1,1). Weights 1/3, 1/18, 1/36.
 */
#ifndef LEDDS_H
#define LEDDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LEDDS_OK 0
#define LEDDS_ERR_INVALID_ARG (-1) /* bad argument or physically invalid parameter      */
#define LEDDS_ERR_CAPACITY (-2)    /* a fixed-capacity buffer overflowed                 */
#define LEDDS_ERR_NAN (-3)         /* non-finite values were detected                    */
#define LEDDS_ERR_TIMEOUT (-4)     /* a bounded device wait gave up                      */
#define LEDDS_ERR_CUDA (-5)        /* a CUDA runtime call failed                         */
#define LEDDS_ERR_STATE (-6)       /* call not valid in the object's current state       */

enum { LEDDS_STORE_F32 = 0, LEDDS_STORE_F16 = 1, LEDDS_STORE_BF16 = 2 };
enum { LEDDS_VOXEL_DISTANCE = 0, LEDDS_VOXEL_SUBDIV = 1 };
enum { LEDDS_LAW_LINEAR = 0, LEDDS_LAW_HERTZ = 1 };
enum { LEDDS_COLLIDE_BGK = 0, LEDDS_COLLIDE_TRT = 1 };
enum { LEDDS_ORIENT_TRIAD = 0, LEDDS_ORIENT_QUAT = 1 };
enum { LEDDS_PATTERN_AB = 0, LEDDS_PATTERN_AA = 1 };
enum { LEDDS_SPHERE = 0, LEDDS_ELLIPSOID = 1 };

/* Sizes fixed at creation. */
typedef struct {
    int nx, ny, nz;          /* lattice nodes; all zero for a DEM-only simulation           */
    double box_lo[3];        /* DEM-only domain (ignored with a lattice)                     */
    double box_hi[3];
    int periodic[3];         /* per axis; a non-periodic axis has a wall on both faces       */
    int max_particles;       /* particle capacity                                            */
    int cand_cap;            /* neighbour-candidate slots per particle (0: 32)               */
    int tile_cap;            /* particle slots per lattice tile (0: 64)                      */
} ledds_dims;

/* Parameters (lattice units). ledds_params_default fills sensible values. */
typedef struct {
    double tau;              /* BGK relaxation time (> 1/2), Sec. 2.3 Eq. (tau)               */
    double fluid_force[3];   /* body force on the fluid (Guo forcing; not in the paper)      */
    int storage;             /* LEDDS_STORE_*: populations stored as f_i - t_i               */
    int storage_scale_log2;  /* 16-bit storage keeps (f_i - t_i) * 2^s                       */
    int voxel;               /* solid fractions of spheres, Sec. 2.4 (ellipsoids: SUBDIV)    */
    int subdiv_n;            /* subdivision sample points per axis (1..16; paper 10)          */
    int law;                 /* contact law, Sec. 2.1 / App. A                               */
    int n_sub;               /* DEM substeps per fluid step, Sec. 2.3                        */
    double rho_f;            /* fluid density used for the analytic buoyancy, Sec. 4.6       */
    double gravity[3];       /* gravity on particles                                         */
    double k_n, k_t;         /* linear-law stiffnesses                                       */
    double young, poisson;   /* Hertz-law material, App. A                                   */
    double restitution;      /* coefficient of restitution, App. A                           */
    double friction;         /* Coulomb coefficient, Eq. (coulombCoeff)                      */
    double skin;             /* neighbour-list skin added to the contact distance            */
    double dem_h;            /* DEM grid spacing, >= largest diameter + skin (needed if any  */
                             /* particles; the grid size is fixed at creation)                */
    int ell_max_iter;        /* ellipsoid common-normal iterations, Sec. 2.1                 */
    double ell_tol;          /* ellipsoid convergence tolerance (fraction of min semi-axis)  */
    int force_fp32;          /* 1: contact forces and torques evaluated in FP32 from FP64    */
                             /* differences and summed in FP64 (contact sets unchanged);     */
                             /* 0: every DEM operation in FP64. Integration is always FP64.  */
    int collision;           /* LEDDS_COLLIDE_BGK (Eq. BGK) or LEDDS_COLLIDE_TRT (Eq. TRT,    */
                             /* 1/tau- = 8 (2 - 1/tau)/(8 - 1/tau)), weighted by 1 - B_tot    */
    int orient;              /* orientation update of the predictor: LEDDS_ORIENT_TRIAD, the  */
                             /* two-stage triad update of Sec. 2.2 with Gram-Schmidt, or      */
                             /* LEDDS_ORIENT_QUAT, the exact rotation by |w| dt about w(t)    */
                             /* through a unit quaternion (agrees with the triad update to    */
                             /* O(dt^3) per step; the triad stays the stored orientation)     */
    int pattern;             /* population arrays: LEDDS_PATTERN_AB, two arrays (pull from   */
                             /* one, write the other), or LEDDS_PATTERN_AA, one array updated */
                             /* in place by alternating steps (half the population memory;   */
                             /* identical results in FP32; not for batch members). Sec. 6     */
                             /* names single-population schemes as a memory reduction        */
    int index64;             /* 1: 64-bit population offsets in the PSM kernel; 0: only when  */
                             /* 19 nx ny nz >= 2^31 (lattices of more than 1.1e8 nodes up to  */
                             /* 2^31 nodes use them automatically; batch members cannot)      */
    int psm_route;           /* PSM kernel loads: 2 staged by the tensor copy engine (TMA) where */
                             /* the lattice suits it (rows a multiple of 16 bytes, nx >= 40   */
                             /* (FP32) / 48 (16-bit), ny >= 8), else direct; 1 always direct  */
                             /* per-thread loads; 0 (default) automatic: staged for FP32      */
                             /* storage, direct for 16-bit storage (the faster of the two on  */
                             /* GB300 for each). All give identical results.                  */
    int ell_screen;          /* 1 (default): before the common-normal iteration, two exact    */
                             /* tests of disjointness (separating plane across the centre line, */
                             /* Perram-Wertheim certificate) skip pairs that cannot touch; 0:   */
                             /* the iteration alone decides, as Sec. 2.1 states the method. The */
                             /* two differ only where the iteration does not converge on a pair */
                             /* the tests prove disjoint (counted in ell_nonconverged).         */
} ledds_params;

/* One particle as given to ledds_set_particles (host memory). */
typedef struct {
    int shape;               /* LEDDS_SPHERE or LEDDS_ELLIPSOID                              */
    double radius;           /* sphere radius (ignored for ellipsoids)                       */
    double semi[3];          /* ellipsoid semi-axes along d1, d2, d3                         */
    double density;          /* particle density (mass = density * volume)                   */
    double pos[3], vel[3], omg[3];
    double triad[9];         /* body axes d1, d2, d3 in world components (orthonormal)       */
} ledds_particle;

/* Device-side error and overflow counters, read by ledds_get_status. */
typedef struct {
    long long steps;         /* fluid steps taken                                            */
    int tile_overflow;       /* particle/tile entries dropped (tile_cap too small)           */
    int cand_overflow;       /* neighbour candidates dropped (cand_cap too small)            */
    int solids_overflow;     /* cell updates that saw more than two solids (kept the top 2)  */
    int skin_violation;      /* a particle moved more than skin/2 between list rebuilds      */
    int ell_nonconverged;    /* ellipsoid contact iterations that hit the cap or missed      */
    int nan_detected;        /* non-finite particle state                                    */
    int n_particles;
    int launches_per_step;   /* kernels launched per fluid step                              */
    int wait_timeout;        /* bounded waits of the staged PSM kernel that gave up (the step's */
                             /* results are then invalid; ledds_get_status returns TIMEOUT)   */
    int psm_staged;          /* 1: the PSM kernel stages its loads with tensor copies          */
} ledds_status;

typedef struct ledds_sim_s* ledds_sim_t;

/* Fill *p with defaults: tau 0.8, FP32 storage, distance voxels (subdiv_n 10), linear law,
 * n_sub 1, rho_f 1, no gravity/force, k_n 1000, k_t 2/7 k_n, restitution 0.7, friction
 * 0.4, skin 0.5, ell_max_iter 60, ell_tol 1e-6, force_fp32 1, BGK collision, triad orientation update, two population arrays, staged PSM route where the lattice suits it, ellipsoid screens on. Returns LEDDS_ERR_INVALID_ARG if p is NULL. */
int ledds_params_default(ledds_params* p);

/* Bytes of device workspace a simulation of these dimensions and parameters needs
 * (populations: 2 x 19 x cells x storage bytes; particles, lists and scratch besides).
 * Errors: INVALID_ARG for NULL pointers, negative sizes or tau <= 1/2. */
int ledds_workspace_size(const ledds_dims* d, const ledds_params* p, size_t* bytes);

/* Create a simulation inside the caller's device workspace (at least
 * ledds_workspace_size bytes, 256-byte aligned) on CUDA stream `stream` (a cudaStream_t,
 * may be 0). The fluid starts at rest with rho = 1; there are no particles.
 * Errors: INVALID_ARG (bad sizes, workspace too small or misaligned), CUDA. */
int ledds_create(const ledds_dims* d, const ledds_params* p, void* d_workspace,
                 size_t bytes, void* stream, ledds_sim_t* out);

/* Release the host-side object (the workspace stays the caller's). */
int ledds_destroy(ledds_sim_t s);

/* Velocity of the wall on face (axis 0..2, side 0 = low, 1 = high): moving-wall
 * bounce-back of Sec. 2.3 (Ladd) for the fluid, surface velocity for DEM contacts. It
 * applies from the next streaming on; the current pre-collision populations are kept.
 * Errors: INVALID_ARG (bad axis/side, or the axis is periodic). */
int ledds_set_wall_velocity(ledds_sim_t s, int axis, int side, const double u[3]);

/* Gravity on the particles (with analytic buoyancy factor 1 - rho_f/rho_p) and the
 * body force on the fluid; either pointer may be NULL to keep the current value. */
int ledds_set_forcing(ledds_sim_t s, const double gravity[3], const double fluid_force[3]);

/* Set the fluid to equilibrium, Eq. (equilibrium), with the given density (cells) and
 * velocity ([3][cells]) device arrays; NULL means rho = 1 or u = 0. */
int ledds_init_fluid(ledds_sim_t s, const float* d_rho, const float* d_u);

/* Set the pre-collision populations directly from a device array [19][cells]. */
int ledds_init_populations(ledds_sim_t s, const float* d_f);

/* Replace all particles with n particles from a host array. Resets accelerations to the
 * buoyant gravity, hydrodynamic forces and contact history to zero. Synchronises.
 * Errors: INVALID_ARG (n > max_particles, non-positive size or density, a particle larger
 * than the DEM grid or periodic box allows, non-orthonormal triad). */
int ledds_set_particles(ledds_sim_t s, int n, const ledds_particle* h_particles);

/* Overwrite positions, velocities, angular velocities and triads of the current n
 * particles from an SoA array of 18*n doubles (see ledds_read_particles) on the host
 * (on_device = 0, synchronises) or the device. Accelerations and history are kept. */
int ledds_write_kinematics(ledds_sim_t s, const double* state, int on_device);

/* Advance n_steps fluid steps (each with n_sub DEM substeps) in the flowchart order of
 * Sec. 3.2. Asynchronous; replays a captured CUDA graph after the first call. */
int ledds_step(ledds_sim_t s, int n_steps);

/* Wait for all work of the simulation's stream. */
int ledds_sync(ledds_sim_t s);

/* Copy the device counters (synchronises). Returns CAPACITY if any overflow counter is
 * non-zero, NAN if non-finite state was seen, else OK; *st is filled in every case. */
int ledds_get_status(ledds_sim_t s, ledds_status* st);

/* Density [cells] and velocity [3][cells] of the current pre-collision populations
 * (Eqs. rho, momentum; with a fluid force, rho u includes half the force). */
int ledds_read_fields(ledds_sim_t s, float* d_rho, float* d_u);

/* Populations [19][cells]: which = 0 the current pre-collision f; which = 1 the stored
 * post-collision array f* of the last step (before streaming). */
int ledds_read_populations(ledds_sim_t s, float* d_f, int which);

/* Particle state [18][n] doubles: pos xyz, vel xyz, omega xyz, triad d1 d2 d3 (9).
 * on_device = 0 copies to host memory and synchronises. */
int ledds_read_particles(ledds_sim_t s, double* state, int on_device);

/* Hydrodynamic force/torque of the last fluid step (Eqs. forceSF, torqueSF) and contact
 * force/torque of the last DEM substep, each [3][n] doubles on the device; any pointer
 * may be NULL. */
int ledds_read_forces(ledds_sim_t s, double* d_Fh, double* d_Mh, double* d_Fc, double* d_Mc);

/* Current contact set (pairs i < j with positive overlap at the current positions) as
 * sorted keys (i << 32 | j) in a device array of capacity cap; *n_out = number of pairs
 * (may exceed cap, then only cap are written). Synchronises. */
int ledds_read_pairs(ledds_sim_t s, uint64_t* d_keys, int cap, int* n_out);

/* Cell keys of the particles at the last neighbour-list rebuild (Sec. 3.2.1) and the
 * particle ids sorted by (key, id); grid_n receives the DEM grid size. Either array
 * may be NULL. Synchronises. */
int ledds_read_cell_keys(ledds_sim_t s, uint32_t* d_keys, int32_t* d_sorted_ids,
                         int grid_n[3]);

/* Solid fractions at the current particle positions: the two largest per cell
 * (d_beta [cells][2], d_ids [cells][2], -1 if absent) and the number of solids touching
 * each cell (d_nsolid [cells]). Sec. 2.4; Sec. 3.2.3 (at most two solids per cell). */
int ledds_voxelize(ledds_sim_t s, float* d_beta, int32_t* d_ids, int32_t* d_nsolid);

/* Profiling: when on, ledds_step launches eagerly and times each stage with CUDA events.
 * ledds_read_profile returns accumulated milliseconds per stage (0 neighbour rebuild,
 * 1 DEM substeps, 2 tile binning, 3 PSM collide-stream, 4 final corrector), the number
 * of profiled steps and of kernel launches, then resets. */
int ledds_set_profiling(ledds_sim_t s, int on);
int ledds_read_profile(ledds_sim_t s, double ms[5], long long* steps, long long* launches);

/* Checkpoint: serialise the full state (populations, particles, contact history, step
 * count) to a host buffer. With h_buf NULL, *bytes receives the size needed. A
 * checkpoint loads into a simulation of the same dims and storage, or of the same dims
 * but larger candidate or tile capacities (the lists are re-laid row by row): that is how
 * a step that overflowed a capacity is replayed with larger capacities. */
int ledds_save(ledds_sim_t s, void* h_buf, size_t* bytes);
int ledds_load(ledds_sim_t s, const void* h_buf, size_t bytes);

/* ------------------------------------------------------------------------------------
 * Batches: many independent simulations (uneven lattices and particle counts) advanced
 * together. Not in the paper; an ensemble form of the same coupled step. Per fluid step
 * the whole batch uses four kernel launches (graph-replayed): a DEM kernel with one CTA
 * per simulation running all substeps, tile binning, one persistent PSM kernel whose
 * CTAs take (simulation, tile) work items from a queue, and the velocity corrector. DEM
 * candidates are found by direct search within each simulation (same contact set as the
 * cell list), so members hold at most 4096 particles.
 * ------------------------------------------------------------------------------------ */
typedef struct ledds_batch_s* ledds_batch_t;

/* Workspace bytes for nsim members described by the arrays dims[nsim], params[nsim]. Every
 * member needs a lattice; all members share the storage format.
 * Errors: INVALID_ARG (as ledds_workspace_size, or a member without a lattice, mixed
 * storage, more than 4096 particles). */
int ledds_batch_workspace_size(int nsim, const ledds_dims* dims, const ledds_params* params,
                               size_t* bytes);

/* Create the batch in a caller-owned workspace of at least ledds_batch_workspace_size
 * bytes (256-byte aligned) on `stream`. Members start with fluid at rest, no particles. */
int ledds_batch_create(int nsim, const ledds_dims* dims, const ledds_params* params,
                       void* d_workspace, size_t bytes, void* stream, ledds_batch_t* out);

/* Handle of member i, valid until ledds_batch_destroy. All single-simulation calls apply
 * to it (walls, forcing, initialisation, particles, reads, status, checkpoint) except
 * ledds_step, ledds_destroy and ledds_read_cell_keys (the batch finds contact candidates
 * by direct search and keeps no cell list), which return LEDDS_ERR_STATE. */
int ledds_batch_sim(ledds_batch_t b, int i, ledds_sim_t* out);

/* Advance every member by n_steps fluid steps (each with its own n_sub DEM substeps).
 * Asynchronous on the batch's stream. */
int ledds_batch_step(ledds_batch_t b, int n_steps);

/* Release the batch and its members' host objects (the workspace stays the caller's). */
int ledds_batch_destroy(ledds_batch_t b);

/* Launch shape of the batched step (BJ config 5's "autotuned tiles"; the paper has no
 * batches): tile_depth planes per lattice tile (8, 16 or 32; tiles are 32 x 8 x depth
 * nodes, one CTA's work item), ctas_per_sm resident PSM CTAs per SM (1 up to the
 * compiled register budget, ledds_batch_get_config of a new batch reports it) and the PSM
 * work order (0 member order, 1 largest members first). Results do not depend on it
 * beyond the order of the hydrodynamic force sums. Default 16, the budget, 0. Errors:
 * INVALID_ARG. */
int ledds_batch_configure(ledds_batch_t b, int tile_depth, int ctas_per_sm, int order);
int ledds_batch_get_config(ledds_batch_t b, int* tile_depth, int* ctas_per_sm, int* order);

/* Autotuner of the batched launch: tries every launch shape (tile depth 8, 16, 32 x
 * resident CTAs per SM x work order), times steps_per_trial steps of each with CUDA events
 * after two warm-up steps, and keeps the fastest. The trial steps are real steps: they
 * advance every member (each candidate computes the same step). The choice is cached
 * for the process by the batch's shape (members' dimensions and particle counts, storage,
 * collision): a later batch of the same shape takes it without trials (and without
 * steps). *choice (may be NULL) receives its index ((depth index x ctas budget + ctas_per_sm
 * - 1) x 2 + order; ledds_batch_get_config gives the values). Synchronous. Errors:
 * INVALID_ARG, CUDA, and those of ledds_batch_step. */
int ledds_batch_autotune(ledds_batch_t b, int steps_per_trial, int* choice);

/* Cell keys and (key, id)-sorted particle ids of the DEM grid, computed without any
 * device allocation. The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory themselves, such as code running under a memory
 * pool that owns the whole device, or a latency-critical path where an allocation could
 * block or fail. It takes no simulation object and no workspace; its scratch (per-cell
 * counts and starts, scan partials, per-particle ranks and scatter order, about 4.2 MB)
 * lives in a fixed array inside the library that every GPU loading the library keeps
 * until the process exits. Cells are ordered in bounded time whatever their occupancy
 * (a grid of one cell included).
 *   d_pos      particle positions on the device, [3][n] doubles (x row, y row, z row)
 *   box_lo/hi  domain; the grid has floor(L/h) cells per axis (at least one), of width
 *              L/cells, exactly as a simulation with dem_h = h builds it
 *   d_keys     output, n cell keys k_x + n_x (k_y + n_y k_z) (device)
 *   d_sorted_ids output, n ids sorted by (key, id) (device)
 *   grid_n     may be NULL; receives the cells per axis
 *   stream     cudaStream_t the work is enqueued on (asynchronous)
 * Limits: at most 262144 grid cells and 262144 particles; larger inputs return
 * LEDDS_ERR_CAPACITY before any device work. Calls on the same device that may overlap
 * (different streams, or host threads without ordering) share one scratch array and must
 * be serialised by the caller; each device has its own copy. The first call in each CUDA
 * context looks up the scratch address (cudaGetSymbolAddress); make that first call
 * before any stream capture. Errors: INVALID_ARG, CAPACITY, CUDA. */
int ledds_cell_list_noalloc(const double* d_pos, int n, const double box_lo[3],
                            const double box_hi[3], double h, uint32_t* d_keys,
                            int32_t* d_sorted_ids, int grid_n[3], void* stream);

const char* ledds_strerror(int code);
int ledds_version(void);

#ifdef __cplusplus
}
#endif
#endif
