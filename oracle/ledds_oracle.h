/*
 * ledds_oracle.h -- plain FP64 CPU oracle of the coupled LBM-PSM-DEM time step of
 * LEDDS (arXiv 2512.04997).
 *
 * TEST INFRASTRUCTURE ONLY. This oracle exists to check the CUDA library against the
 * paper. Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it. The product library never calls it and shares no code, header, table or
 * constant with it.
 *
 * Every function follows the paper section or equation named in its comment, in the
 * paper's order, with no blocking, fusion or reordering. Floating point is IEEE FP64
 * (compiled with -ffp-contract=off) except the subdivision inside/outside predicate,
 * which decides an integer count and is therefore evaluated in FP32 exactly as the
 * GPU kernel evaluates it (see or_subdiv_count).
 */
#ifndef LEDDS_ORACLE_H
#define LEDDS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Shapes, voxelisation methods and contact laws. */
enum { OR_SPHERE = 0, OR_ELLIPSOID = 1 };
enum { OR_VOXEL_DISTANCE = 0, OR_VOXEL_SUBDIV = 1 };
enum { OR_LAW_LINEAR = 0, OR_LAW_HERTZ = 1 };
enum { OR_COLLIDE_BGK = 0, OR_COLLIDE_TRT = 1 };
enum { OR_ORIENT_TRIAD = 0, OR_ORIENT_QUAT = 1 };

typedef struct {
    double tau;             /* BGK relaxation time, Eq. (tau)                                */
    double fluid_force[3];  /* constant body force on the fluid (Guo forcing); 0 = off        */
    int voxel;              /* OR_VOXEL_DISTANCE (Eq. naiveSolidFrac) or OR_VOXEL_SUBDIV      */
    int subdiv_n;           /* sample points per axis of the subdivision method (paper: 10)   */
    int law;                /* OR_LAW_LINEAR or OR_LAW_HERTZ (App. A)                         */
    int n_sub;              /* DEM substeps per fluid step (Sec. 2.3, last paragraph)         */
    double rho_f;           /* fluid density for the analytic buoyancy (Sec. 4.6)             */
    double gravity[3];      /* gravity acting on the particles                                */
    double k_n, k_t;        /* linear-law stiffnesses                                         */
    double young, poisson;  /* Hertz-law material (App. A)                                    */
    double restitution;     /* coefficient of restitution epsilon (App. A)                    */
    double friction;        /* Coulomb coefficient mu, Eq. (coulombCoeff)                     */
    double dem_h;           /* requested DEM grid spacing (>= largest particle diameter)      */
    int ell_max_iter;       /* common-normal iteration cap (Sec. 2.1)                         */
    double ell_tol;         /* common-normal convergence tolerance, relative to min semi-axis */
    int collision;          /* OR_COLLIDE_BGK (Eq. BGK) or OR_COLLIDE_TRT (Eq. TRT)            */
    int orient;             /* OR_ORIENT_TRIAD (Sec. 2.2 triad update) or OR_ORIENT_QUAT      */
} or_params;

typedef struct or_sim or_sim;

/*
 * Create an oracle simulation.
 *   nx,ny,nz  lattice size; all zero for a DEM-only simulation.
 *   box_lo/hi DEM domain for DEM-only runs (ignored with a lattice, whose domain is
 *             [-1/2, n-1/2] on each axis: nodes sit at integers, walls halfway).
 *   periodic  per axis; a non-periodic axis has a wall on each face.
 *   u_wall    [axis][side][component], side 0 = low face, 1 = high face.
 *   max_particles capacity.
 */
or_sim* or_create(int nx, int ny, int nz, const double box_lo[3], const double box_hi[3],
                  const int periodic[3], const double u_wall[18], const or_params* p,
                  int max_particles);
void or_destroy(or_sim* s);

/* Fluid state. Layout of field arrays: cell index x + nx*(y + ny*z). */
void or_init_equilibrium(or_sim* s, const double* rho, const double* u3); /* NULL => rho=1,u=0 */
void or_set_populations(or_sim* s, const double* f);   /* f[i*N + cell], pre-collision       */
void or_get_populations(const or_sim* s, double* f);   /* f[i*N + cell], pre-collision       */
void or_moments(const or_sim* s, double* rho, double* u3);  /* u3[a*N + cell]               */
void or_equilibrium(double rho, const double u[3], double feq[19]);  /* Eq. (equilibrium)   */
void or_lattice_tables(int c[57], double w[19], int opp[19]);        /* D3Q19 tables         */

/* Particles. Arrays are per particle, xyz-contiguous; triad = d1,d2,d3 (rows of R). */
int or_set_particles(or_sim* s, int n, const int* shape, const double* radius,
                     const double* semi, const double* density, const double* pos,
                     const double* vel, const double* omg, const double* triad);
void or_get_particles(const or_sim* s, double* pos, double* vel, double* omg, double* triad);
void or_get_forces(const or_sim* s, double* Fh, double* Mh, double* Fc, double* Mc);
void or_get_accel(const or_sim* s, double* acc, double* alpha);
/* Unit quaternion (w, x, y, z) of the body-to-world rotation whose columns are the
 * triad d1, d2, d3 (Shepperd's method); and the triad of a unit quaternion. */
void or_quat_from_triad(const double triad[9], double q[4]);
/* Solid weight B_k of a solid fraction beta, Eq. (bk). */
double or_bk(double beta, double tau);
void or_triad_from_quat(const double q[4], double triad[9]);

/* One coupled (or DEM-only) time step, flowchart order of Sec. 3.2. */
void or_step(or_sim* s, int nsteps);

/* Unit-level entry points used by the tests. */
void or_voxelize(or_sim* s, double* beta2, int* id2, int* nsolid);    /* top-2 per cell */
void or_lbm_psm_step(or_sim* s);                /* Table 1 PSM rows at current particle state */
int  or_cell_keys(or_sim* s, unsigned* keys, int* sorted_ids, int grid_n[3]);
int  or_contacts(or_sim* s, long long* pair_keys, int cap);   /* current contact set (i<j)  */
void or_contact_forces(or_sim* s, double dt);                 /* Fc, Mc at current state    */
int  or_subdiv_count(const double rel[3], int shape, double radius, const double semi[3],
                     const double triad[9], int n);
double or_beta_distance(const double rel[3], double radius);
void or_cell_collide(const double f[19], double tau, int collision, const double force[3], int ns,
                     const double* B, const double* uk, const double* arm,
                     double fstar[19], double* Fk, double* Mk);
int  or_ellipsoid_contact(const double ri[3], const double Ri[9], const double si[3],
                          const double rj[3], const double Rj[9], const double sj[3],
                          int max_iter, double tol, double* delta, double en[3],
                          double cp[3], double* rho_i, double* rho_j, int* iters);
/* 1 if a Perram-Wertheim certificate shows the two ellipsoids disjoint (F(l) > 1 + 1e-9
 * at one of at most 16 golden-section points), else 0. */
void or_solids_at(const or_sim* s, int x, int y, int z, int ids[2], double beta[2], int* total);
int  or_threads(void); /* 1, or the OpenMP team size of the timing build */
int  or_pw_separated(const double ri[3], const double Ri[9], const double si[3],
                     const double rj[3], const double Rj[9], const double sj[3]);
void or_status(const or_sim* s, long long out[4]); /* solids overflow, ell nonconv, ... */

#ifdef __cplusplus
}
#endif
#endif
