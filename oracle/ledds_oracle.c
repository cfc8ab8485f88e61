/*
 * ledds_oracle.c -- plain FP64 CPU oracle of the coupled LBM-PSM-DEM step of LEDDS
 * (arXiv 2512.04997).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's CPU
 * baseline. The CUDA library never calls it, and the two share no code.
 *
 * The code is deliberately slow and literal. Each function names the paper passage it
 * follows; where the paper is silent or garbled, the reading taken is stated at the
 * place it is used. Build: gcc -O2 -ffp-contract=off -fPIC -shared.
 */
#include "ledds_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------ */
/* D3Q19 lattice (Sec. 2.3; weights are the textbook ones the paper refers to).          */
/* Velocity order: rest; +x,-x,+y,-y,+z,-z; then the 12 edge velocities, each followed  */
/* by its opposite.                                                                       */
/* ------------------------------------------------------------------------------------ */
static const int CV[19][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double TW(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
static int OPP(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

/* Threads the lattice update runs on: 1 in the parity build, the OpenMP team size in the
 * build used for the timed CPU baseline. */
int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_lattice_tables(int c[57], double w[19], int opp[19]) {
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = CV[i][a];
        w[i] = TW(i);
        opp[i] = OPP(i);
    }
}

/* Eq. (equilibrium): second-order Hermite equilibrium with c_s^2 = 1/3. */
void or_equilibrium(double rho, const double u[3], double feq[19]) {
    const double cs2 = 1.0 / 3.0;
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        feq[i] = rho * TW(i) *
                 (1.0 + cu / cs2 + (cu * cu) / (2.0 * cs2 * cs2) - usq / (2.0 * cs2));
    }
}

/* ------------------------------------------------------------------------------------ */
/* Simulation object                                                                      */
/* ------------------------------------------------------------------------------------ */
struct or_sim {
    or_params p;
    int nx, ny, nz;          /* lattice (0 => DEM only) */
    long long ncell;
    int periodic[3];
    double u_wall[3][2][3];
    double lo[3], hi[3], L[3];
    double *f, *fn;          /* f[cell*19 + i], pre-collision */
    /* particles */
    int n, cap;
    int* shape;
    double *radius, *semi, *bound, *rho_p, *mass, *inertia;
    double *pos, *vel, *omg, *acc, *alpha, *triad;
    double *Fc, *Mc, *Fh, *Mh, *Fh_prev, *Mh_prev;
    /* contact list of the previous substep, sorted by (i,j), with tangential history */
    int ncont, contcap;
    int *ci, *cj;
    double* chist;
    double* whist;          /* [particle][face 0..5][3] wall tangential history */
    /* DEM grid */
    int gn[3];
    double gh[3];
    long long nsolid_overflow;
    long long ell_nonconverged;
    long long steps;
};

static void vcross(const double a[3], const double b[3], double o[3]) {
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}
static double vdot(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static double vnorm(const double a[3]) { return sqrt(vdot(a, a)); }

static void* xcalloc(size_t n, size_t s) {
    void* p = calloc(n ? n : 1, s);
    if (!p) abort();
    return p;
}

or_sim* or_create(int nx, int ny, int nz, const double box_lo[3], const double box_hi[3],
                  const int periodic[3], const double u_wall[18], const or_params* p,
                  int max_particles) {
    or_sim* s = (or_sim*)xcalloc(1, sizeof(or_sim));
    s->p = *p;
    s->nx = nx; s->ny = ny; s->nz = nz;
    s->ncell = (long long)nx * ny * nz;
    for (int a = 0; a < 3; ++a) s->periodic[a] = periodic[a];
    for (int a = 0; a < 3; ++a)
        for (int e = 0; e < 2; ++e)
            for (int c = 0; c < 3; ++c) s->u_wall[a][e][c] = u_wall[6 * a + 3 * e + c];
    int n3[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        if (s->ncell > 0) {
            /* Nodes sit at integer positions and own the cell [x-1/2, x+1/2]; walls are
             * halfway between the last node and the first solid node. */
            s->lo[a] = -0.5;
            s->hi[a] = n3[a] - 0.5;
        } else {
            s->lo[a] = box_lo[a];
            s->hi[a] = box_hi[a];
        }
        s->L[a] = s->hi[a] - s->lo[a];
    }
    if (s->ncell > 0) {
        s->f = (double*)xcalloc((size_t)s->ncell * 19, sizeof(double));
        s->fn = (double*)xcalloc((size_t)s->ncell * 19, sizeof(double));
        or_init_equilibrium(s, NULL, NULL);
    }
    int c = max_particles > 0 ? max_particles : 1;
    s->cap = c;
    s->shape = (int*)xcalloc(c, sizeof(int));
    s->radius = (double*)xcalloc(c, sizeof(double));
    s->bound = (double*)xcalloc(c, sizeof(double));
    s->semi = (double*)xcalloc(3 * c, sizeof(double));
    s->rho_p = (double*)xcalloc(c, sizeof(double));
    s->mass = (double*)xcalloc(c, sizeof(double));
    s->inertia = (double*)xcalloc(3 * c, sizeof(double));
    s->pos = (double*)xcalloc(3 * c, sizeof(double));
    s->vel = (double*)xcalloc(3 * c, sizeof(double));
    s->omg = (double*)xcalloc(3 * c, sizeof(double));
    s->acc = (double*)xcalloc(3 * c, sizeof(double));
    s->alpha = (double*)xcalloc(3 * c, sizeof(double));
    s->triad = (double*)xcalloc(9 * c, sizeof(double));
    s->Fc = (double*)xcalloc(3 * c, sizeof(double));
    s->Mc = (double*)xcalloc(3 * c, sizeof(double));
    s->Fh = (double*)xcalloc(3 * c, sizeof(double));
    s->Mh = (double*)xcalloc(3 * c, sizeof(double));
    s->Fh_prev = (double*)xcalloc(3 * c, sizeof(double));
    s->Mh_prev = (double*)xcalloc(3 * c, sizeof(double));
    s->whist = (double*)xcalloc(18 * c, sizeof(double));
    s->contcap = 16;
    s->ci = (int*)xcalloc(s->contcap, sizeof(int));
    s->cj = (int*)xcalloc(s->contcap, sizeof(int));
    s->chist = (double*)xcalloc(3 * s->contcap, sizeof(double));
    /* DEM grid (Sec. 3.2.1): spacing >= the requested h, integer cells per axis. */
    for (int a = 0; a < 3; ++a) {
        int g = p->dem_h > 0.0 ? (int)floor(s->L[a] / p->dem_h) : 1;
        if (g < 1) g = 1;
        s->gn[a] = g;
        s->gh[a] = s->L[a] / g;
    }
    return s;
}

void or_destroy(or_sim* s) {
    if (!s) return;
    free(s->f); free(s->fn);
    free(s->shape); free(s->radius); free(s->bound); free(s->semi); free(s->rho_p);
    free(s->mass); free(s->inertia); free(s->pos); free(s->vel); free(s->omg);
    free(s->acc); free(s->alpha); free(s->triad); free(s->Fc); free(s->Mc);
    free(s->Fh); free(s->Mh); free(s->Fh_prev); free(s->Mh_prev); free(s->whist);
    free(s->ci); free(s->cj); free(s->chist);
    free(s);
}

/* ------------------------------------------------------------------------------------ */
/* Fluid state                                                                            */
/* ------------------------------------------------------------------------------------ */

/* Initialisation f = f^eq(rho, u) (Sec. 2.3, end). */
void or_init_equilibrium(or_sim* s, const double* rho, const double* u3) {
    for (long long c = 0; c < s->ncell; ++c) {
        double r = rho ? rho[c] : 1.0;
        double u[3] = {0, 0, 0};
        if (u3)
            for (int a = 0; a < 3; ++a) u[a] = u3[a * s->ncell + c];
        or_equilibrium(r, u, s->f + 19 * c);
    }
}

void or_set_populations(or_sim* s, const double* f) {
    for (long long c = 0; c < s->ncell; ++c)
        for (int i = 0; i < 19; ++i) s->f[19 * c + i] = f[i * s->ncell + c];
}

void or_get_populations(const or_sim* s, double* f) {
    for (long long c = 0; c < s->ncell; ++c)
        for (int i = 0; i < 19; ++i) f[i * s->ncell + c] = s->f[19 * c + i];
}

/* Eqs. (rho), (momentum). With a fluid body force F the velocity carries the usual
 * half-force shift of Guo forcing: rho u = sum f c + F/2. */
static void cell_moments(const double* f, const double F[3], double* rho, double u[3]) {
    double r = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < 19; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += f[i] * CV[i][a];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / r;
}

void or_moments(const or_sim* s, double* rho, double* u3) {
    for (long long c = 0; c < s->ncell; ++c) {
        double r, u[3];
        cell_moments(s->f + 19 * c, s->p.fluid_force, &r, u);
        rho[c] = r;
        for (int a = 0; a < 3; ++a) u3[a * s->ncell + c] = u[a];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Particles                                                                              */
/* ------------------------------------------------------------------------------------ */

/* Gram-Schmidt re-orthonormalisation of the triad (the paper is silent; reading: d1
 * normalised, d2 orthogonalised to d1 and normalised, d3 = d1 x d2). */
static void orthonormalise(double* d) {
    double* d1 = d;
    double* d2 = d + 3;
    double* d3 = d + 6;
    double n1 = vnorm(d1);
    for (int a = 0; a < 3; ++a) d1[a] /= n1;
    double p = vdot(d2, d1);
    for (int a = 0; a < 3; ++a) d2[a] -= p * d1[a];
    double n2 = vnorm(d2);
    for (int a = 0; a < 3; ++a) d2[a] /= n2;
    vcross(d1, d2, d3);
}

int or_set_particles(or_sim* s, int n, const int* shape, const double* radius,
                     const double* semi, const double* density, const double* pos,
                     const double* vel, const double* omg, const double* triad) {
    if (n > s->cap) return -1;
    s->n = n;
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < n; ++k) {
        s->shape[k] = shape[k];
        s->rho_p[k] = density[k];
        double V;
        if (shape[k] == OR_SPHERE) {
            double R = radius[k];
            s->radius[k] = R;
            s->bound[k] = R;
            for (int a = 0; a < 3; ++a) s->semi[3 * k + a] = R;
            V = 4.0 / 3.0 * pi * R * R * R;
            s->mass[k] = density[k] * V;
            /* Sphere inertia, Sec. 2.2. */
            for (int a = 0; a < 3; ++a) s->inertia[3 * k + a] = 2.0 * s->mass[k] * R * R / 5.0;
        } else {
            double A = semi[3 * k], B = semi[3 * k + 1], C = semi[3 * k + 2];
            for (int a = 0; a < 3; ++a) s->semi[3 * k + a] = semi[3 * k + a];
            double mx = A > B ? A : B;
            mx = mx > C ? mx : C;
            s->radius[k] = mx;
            s->bound[k] = mx;
            V = 4.0 / 3.0 * pi * A * B * C;
            s->mass[k] = density[k] * V;
            /* Ellipsoid inertia about the body axes d1, d2, d3, Sec. 2.2. */
            s->inertia[3 * k + 0] = s->mass[k] * (B * B + C * C) / 5.0;
            s->inertia[3 * k + 1] = s->mass[k] * (A * A + C * C) / 5.0;
            s->inertia[3 * k + 2] = s->mass[k] * (A * A + B * B) / 5.0;
        }
        for (int a = 0; a < 3; ++a) {
            s->pos[3 * k + a] = pos[3 * k + a];
            s->vel[3 * k + a] = vel[3 * k + a];
            s->omg[3 * k + a] = omg[3 * k + a];
            s->alpha[3 * k + a] = 0.0;
            s->Fc[3 * k + a] = s->Mc[3 * k + a] = 0.0;
            s->Fh[3 * k + a] = s->Mh[3 * k + a] = 0.0;
            s->Fh_prev[3 * k + a] = s->Mh_prev[3 * k + a] = 0.0;
            /* Initial acceleration: gravity reduced by the analytic buoyancy of Sec. 4.6. */
            s->acc[3 * k + a] = s->p.gravity[a] * (1.0 - s->p.rho_f / density[k]);
        }
        for (int m = 0; m < 9; ++m) s->triad[9 * k + m] = triad[9 * k + m];
        for (int m = 0; m < 18; ++m) s->whist[18 * k + m] = 0.0;
    }
    s->ncont = 0;
    return 0;
}

void or_get_particles(const or_sim* s, double* pos, double* vel, double* omg, double* triad) {
    memcpy(pos, s->pos, sizeof(double) * 3 * s->n);
    memcpy(vel, s->vel, sizeof(double) * 3 * s->n);
    memcpy(omg, s->omg, sizeof(double) * 3 * s->n);
    memcpy(triad, s->triad, sizeof(double) * 9 * s->n);
}

void or_get_forces(const or_sim* s, double* Fh, double* Mh, double* Fc, double* Mc) {
    memcpy(Fh, s->Fh, sizeof(double) * 3 * s->n);
    memcpy(Mh, s->Mh, sizeof(double) * 3 * s->n);
    memcpy(Fc, s->Fc, sizeof(double) * 3 * s->n);
    memcpy(Mc, s->Mc, sizeof(double) * 3 * s->n);
}

void or_get_accel(const or_sim* s, double* acc, double* alpha) {
    memcpy(acc, s->acc, sizeof(double) * 3 * s->n);
    memcpy(alpha, s->alpha, sizeof(double) * 3 * s->n);
}

void or_status(const or_sim* s, long long out[4]) {
    out[0] = s->nsolid_overflow;
    out[1] = s->ell_nonconverged;
    out[2] = s->steps;
    out[3] = s->ncont;
}

/* Minimum-image displacement on periodic axes (positions are kept inside the box). */
static double min_image(const or_sim* s, int a, double d) {
    if (s->periodic[a]) {
        if (d > 0.5 * s->L[a]) d -= s->L[a];
        else if (d < -0.5 * s->L[a]) d += s->L[a];
    }
    return d;
}

/* ------------------------------------------------------------------------------------ */
/* Solid fractions (Sec. 2.4)                                                             */
/* ------------------------------------------------------------------------------------ */

/* Distance-based method, Eq. (naiveSolidFrac): overlap of the sphere with a sphere of
 * volume dx^3 centred on the node. rel = node - particle centre. */
double or_beta_distance(const double rel[3], double radius) {
    const double pi = 3.14159265358979323846;
    double Rc = cbrt(3.0 / (4.0 * pi));
    double d = vnorm(rel);
    double dsc = radius + Rc - d;
    if (dsc < 0.0) return 0.0;
    if (dsc > 2.0 * Rc) return 1.0;
    return dsc / (2.0 * Rc);
}

/* Subdivision method (Sec. 2.4): count of n^3 points evenly spread inside the cell that
 * lie strictly inside the solid. The paper prints |r_j - s_i| < R_k, where r_j would be
 * the cell centre; reading: the sample point's distance to the particle centre r_k.
 * Sample offsets from the node are (2m+1-n)/(2n), m = 0..n-1 on each axis.
 * The predicate decides an integer, so it is evaluated in FP32 in exactly the order the
 * GPU kernel uses: rel (FP64 node-minus-centre, minimum image) rounded to FP32;
 * d = rel + offset; sphere: ((dx*dx + dy*dy) + dz*dz) < fl32(R*R);
 * ellipsoid: q_j = (m_j0*dx + m_j1*dy) + m_j2*dz with m_jc = fl32(d_j[c]/semi_j),
 * inside iff ((q0*q0 + q1*q1) + q2*q2) < 1. */
int or_subdiv_count(const double rel[3], int shape, double radius, const double semi[3],
                    const double triad[9], int n) {
    float px = (float)rel[0], py = (float)rel[1], pz = (float)rel[2];
    float m[3][3] = {{0.0f}};
    float R2 = (float)(radius * radius);
    if (shape == OR_ELLIPSOID)
        for (int j = 0; j < 3; ++j)
            for (int c = 0; c < 3; ++c) m[j][c] = (float)(triad[3 * j + c] / semi[j]);
    int count = 0;
    for (int a = 0; a < n; ++a) {
        float oa = (float)(2 * a + 1 - n) / (float)(2 * n);
        for (int b = 0; b < n; ++b) {
            float ob = (float)(2 * b + 1 - n) / (float)(2 * n);
            for (int c = 0; c < n; ++c) {
                float oc = (float)(2 * c + 1 - n) / (float)(2 * n);
                float dx = px + oa, dy = py + ob, dz = pz + oc;
                if (shape == OR_SPHERE) {
                    float s2 = (dx * dx + dy * dy) + dz * dz;
                    if (s2 < R2) ++count;
                } else {
                    float q0 = (m[0][0] * dx + m[0][1] * dy) + m[0][2] * dz;
                    float q1 = (m[1][0] * dx + m[1][1] * dy) + m[1][2] * dz;
                    float q2 = (m[2][0] * dx + m[2][1] * dy) + m[2][2] * dz;
                    float s2 = (q0 * q0 + q1 * q1) + q2 * q2;
                    if (s2 < 1.0f) ++count;
                }
            }
        }
    }
    return count;
}

/* Solid fraction of particle k at node rel = node - r_k. Spheres follow the configured
 * method; ellipsoids always use subdivision (the distance method is for spheres only,
 * Sec. 2.4). */
static double beta_of(const or_sim* s, int k, const double rel[3]) {
    if (s->shape[k] == OR_SPHERE && s->p.voxel == OR_VOXEL_DISTANCE)
        return or_beta_distance(rel, s->radius[k]);
    int n = s->p.subdiv_n;
    int cnt = or_subdiv_count(rel, s->shape[k], s->radius[k], s->semi + 3 * k,
                              s->triad + 9 * k, n);
    return (double)cnt / ((double)n * n * n);
}

/* Per-cell solid list: at most two solids (k = 2, Sec. 3.2.3). The paper does not say
 * which two to keep when more touch a cell; reading: the two largest beta, ties to the
 * lower particle id; the excess is counted. */
typedef struct {
    int ns;
    int id[2];
    double beta[2];
    int total;
} cell_solids;

static void solids_insert(cell_solids* cs, int k, double b) {
    cs->total++;
    /* ordered by (beta desc, id asc) */
    if (cs->ns < 2) {
        cs->id[cs->ns] = k;
        cs->beta[cs->ns] = b;
        cs->ns++;
    } else {
        int worst = 1;
        int better = (b > cs->beta[worst]) || (b == cs->beta[worst] && k < cs->id[worst]);
        if (!better) return;
        cs->id[worst] = k;
        cs->beta[worst] = b;
    }
    if (cs->ns == 2) {
        int swap = (cs->beta[1] > cs->beta[0]) ||
                   (cs->beta[1] == cs->beta[0] && cs->id[1] < cs->id[0]);
        if (swap) {
            int ti = cs->id[0]; cs->id[0] = cs->id[1]; cs->id[1] = ti;
            double tb = cs->beta[0]; cs->beta[0] = cs->beta[1]; cs->beta[1] = tb;
        }
    }
}

/* Table 1, "Compute solid fractions": for each particle, every node in its bounding box
 * (one lattice unit of margin) gets its solid fraction; each node keeps its top two. */
static cell_solids* compute_solids(const or_sim* s) {
    cell_solids* cs = (cell_solids*)xcalloc((size_t)s->ncell, sizeof(cell_solids));
    int n3[3] = {s->nx, s->ny, s->nz};
    for (int k = 0; k < s->n; ++k) {
        const double* r = s->pos + 3 * k;
        double e = s->bound[k] + 1.0;
        int lo[3], hi[3];
        if (!(isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]))) continue;
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int)ceil(r[a] - e);
            hi[a] = (int)floor(r[a] + e);
        }
        for (int z = lo[2]; z <= hi[2]; ++z)
            for (int y = lo[1]; y <= hi[1]; ++y)
                for (int x = lo[0]; x <= hi[0]; ++x) {
                    int q[3] = {x, y, z};
                    int ok = 1;
                    for (int a = 0; a < 3; ++a) {
                        if (s->periodic[a]) {
                            q[a] %= n3[a];
                            if (q[a] < 0) q[a] += n3[a];
                        } else if (q[a] < 0 || q[a] >= n3[a]) {
                            ok = 0;
                        }
                    }
                    if (!ok) continue;
                    double rel[3];
                    for (int a = 0; a < 3; ++a) rel[a] = min_image(s, a, (double)q[a] - r[a]);
                    double b = beta_of(s, k, rel);
                    if (b > 0.0) {
                        long long c = q[0] + (long long)s->nx * (q[1] + (long long)s->ny * q[2]);
                        solids_insert(&cs[c], k, b);
                    }
                }
    }
    return cs;
}

/* The solids of one node as compute_solids finds them (the same particle order, the same
 * bounding boxes with their periodic images, the same top-two selection), for spot checks
 * on lattices too large to voxelise whole. A periodic axis counts every image of the
 * node inside a particle's box, as the box loop does. */
void or_solids_at(const or_sim* s, int x, int y, int z, int ids[2], double beta[2], int* total) {
    cell_solids cs;
    memset(&cs, 0, sizeof(cs));
    int n3[3] = {s->nx, s->ny, s->nz};
    int node[3] = {x, y, z};
    for (int k = 0; k < s->n; ++k) {
        const double* r = s->pos + 3 * k;
        double e = s->bound[k] + 1.0;
        if (!(isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]))) continue;
        long long mult = 1;
        for (int a = 0; a < 3; ++a) {
            long long lo = (long long)ceil(r[a] - e), hi = (long long)floor(r[a] + e);
            long long m;
            if (s->periodic[a]) {
                /* integers q in [lo, hi] with q = node (mod n) */
                long long n = n3[a];
                long long first = (long long)ceil((double)(lo - node[a]) / (double)n);
                long long last = (long long)floor((double)(hi - node[a]) / (double)n);
                m = last >= first ? last - first + 1 : 0;
            } else {
                m = (lo <= node[a] && node[a] <= hi) ? 1 : 0;
            }
            mult *= m;
        }
        if (mult == 0) continue;
        double rel[3];
        for (int a = 0; a < 3; ++a) rel[a] = min_image(s, a, (double)node[a] - r[a]);
        double b = beta_of(s, k, rel);
        if (b > 0.0)
            for (long long q = 0; q < mult; ++q) solids_insert(&cs, k, b);
    }
    for (int m = 0; m < 2; ++m) {
        ids[m] = m < cs.ns ? cs.id[m] : -1;
        beta[m] = m < cs.ns ? cs.beta[m] : 0.0;
    }
    *total = cs.total;
}

void or_voxelize(or_sim* s, double* beta2, int* id2, int* nsolid) {
    cell_solids* cs = compute_solids(s);
    for (long long c = 0; c < s->ncell; ++c) {
        for (int m = 0; m < 2; ++m) {
            beta2[2 * c + m] = m < cs[c].ns ? cs[c].beta[m] : 0.0;
            id2[2 * c + m] = m < cs[c].ns ? cs[c].id[m] : -1;
        }
        nsolid[c] = cs[c].total;
    }
    free(cs);
}

/* ------------------------------------------------------------------------------------ */
/* PSM collision of one cell (Sec. 2.4)                                                   */
/* ------------------------------------------------------------------------------------ */

/* One cell's collision with partially saturated solids, Eqs. (psm1), (lbePS):
 *   f*_i = f_i + (1 - B_tot) Omega^fluid_i + sum_k B_k Omega^s_{i,k}
 * with Omega^fluid the BGK operator, Eq. (BGK), or the TRT operator, Eq. (TRT):
 *   f+_i = (f_i + f_ibar)/2, f-_i = (f_i - f_ibar)/2 (Eq. trt_populations), the same split
 *   of f^eq, Omega^TRT_i = -(1/tau+) (f+_i - feq+_i) - (1/tau-) (f-_i - feq-_i),
 *   tau+ = tau and 1/tau- = 8 (2 - 1/tau+) / (8 - 1/tau+);
 * the solid operator
 *   Omega^s_{i,k} = [f_ibar - f^eq_ibar(rho,u)] - [f_i - f^eq_i(rho,u_k)],
 * B_tot = min(sum_k B_k, 1) (Eq. btot) and the hydrodynamic force and torque of
 * Eqs. (forceSF), (torqueSF) for this cell (dx^3/dt = 1 in lattice units):
 *   F_k = -B_k sum_i Omega^s_{i,k} c_i,  M_k = -B_k arm_k x sum_i Omega^s_{i,k} c_i.
 * The paper does not renormalise B_k when their sum exceeds one; reading: as written.
 * A fluid body force (not part of the paper; Guo forcing) adds (1 - B_tot) times
 *   BGK: (1 - 1/(2 tau)) t_i [3 (c_i - u) + 9 (c_i.u) c_i] . F,
 *   TRT: the part even in c_i, t_i [-3 u + 9 (c_i.u) c_i] . F, times (1 - 1/(2 tau+)) and
 *        the part odd in c_i, t_i 3 c_i . F, times (1 - 1/(2 tau-)) (reading).
 * B[k], uk[3k..], arm[3k..] describe the ns <= 2 solids. */
void or_cell_collide(const double f[19], double tau, int collision, const double force[3], int ns,
                     const double* B, const double* uk, const double* arm,
                     double fstar[19], double* Fk, double* Mk) {
    double rho, u[3];
    cell_moments(f, force, &rho, u);
    double feq[19];
    or_equilibrium(rho, u, feq);
    double Btot = 0.0;
    for (int k = 0; k < ns; ++k) Btot += B[k];
    if (Btot > 1.0) Btot = 1.0;
    const double wp = 1.0 / tau;                       /* 1/tau+ */
    const double wm = 8.0 * (2.0 - wp) / (8.0 - wp);   /* 1/tau- */
    double fs[19];
    for (int i = 0; i < 19; ++i) {
        const int o = OPP(i);
        double om;
        if (collision == OR_COLLIDE_TRT) {
            const double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
            const double ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
            om = -wp * (fp - ep) - wm * (fm - em);
        } else {
            om = -(1.0 / tau) * (f[i] - feq[i]);
        }
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        double even = 0.0, odd = 0.0;
        for (int a = 0; a < 3; ++a) {
            even += (-3.0 * u[a] + 9.0 * cu * CV[i][a]) * force[a];
            odd += 3.0 * CV[i][a] * force[a];
        }
        double guo;
        if (collision == OR_COLLIDE_TRT)
            guo = TW(i) * ((1.0 - 0.5 * wp) * even + (1.0 - 0.5 * wm) * odd);
        else
            guo = TW(i) * (1.0 - 0.5 / tau) * (even + odd);
        fs[i] = f[i] + (1.0 - Btot) * (om + guo);
    }
    for (int k = 0; k < ns; ++k) {
        double feqk[19];
        or_equilibrium(rho, uk + 3 * k, feqk);
        double sc[3] = {0, 0, 0};
        for (int i = 0; i < 19; ++i) {
            int o = OPP(i);
            double oms = (f[o] - feq[o]) - (f[i] - feqk[i]);
            fs[i] += B[k] * oms;
            for (int a = 0; a < 3; ++a) sc[a] += oms * CV[i][a];
        }
        double cr[3];
        vcross(arm + 3 * k, sc, cr);
        for (int a = 0; a < 3; ++a) {
            Fk[3 * k + a] = -B[k] * sc[a];
            Mk[3 * k + a] = -B[k] * cr[a];
        }
    }
    for (int i = 0; i < 19; ++i) fstar[i] = fs[i];
}

/* Eq. (bk). */
static double Bk_of(double beta, double tau) {
    return beta * (tau - 0.5) / ((1.0 - beta) + (tau - 0.5));
}

double or_bk(double beta, double tau) { return Bk_of(beta, tau); }

/* ------------------------------------------------------------------------------------ */
/* PSM fluid update: Table 1 "PSM fluid-particle coupling" and "Force reduction" rows.   */
/* Solid fractions at the current particle positions, collision of every cell, then     */
/* streaming (Eq. collAndStream) with halfway bounce-back at walls (velocity-modified    */
/* for moving walls, Sec. 2.3, Ladd), then per-particle force sums.                       */
/* ------------------------------------------------------------------------------------ */
void or_lbm_psm_step(or_sim* s) {
    const double cs2 = 1.0 / 3.0;
    cell_solids* cs = compute_solids(s);
    for (int k = 0; k < s->n; ++k)
        for (int a = 0; a < 3; ++a) s->Fh[3 * k + a] = s->Mh[3 * k + a] = 0.0;
    long long over = 0;
    int n3[3] = {s->nx, s->ny, s->nz};
    /* The timed CPU baseline builds this file a second time with OpenMP: planes are
     * collided and streamed in parallel (every streamed slot has exactly one source), and
     * the per-particle sums become atomic additions (their order then varies, so that
     * build is used for timing only; the parity build has no OpenMP and runs in order). */
#pragma omp parallel for schedule(static) reduction(+ : over)
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long long c = x + (long long)s->nx * (y + (long long)s->ny * z);
                const double* f = s->f + 19 * c;
                int ns = cs[c].ns;
                if (cs[c].total > 2) over++;
                double B[2], uk[6], arm[6], Fk[6], Mk[6];
                for (int m = 0; m < ns; ++m) {
                    int k = cs[c].id[m];
                    B[m] = Bk_of(cs[c].beta[m], s->p.tau);
                    double node[3] = {(double)x, (double)y, (double)z};
                    for (int a = 0; a < 3; ++a)
                        arm[3 * m + a] = min_image(s, a, node[a] - s->pos[3 * k + a]);
                    /* Solid surface velocity. The paper prints u_k = v_k - w_k x (r_j - r_k);
                     * that sign contradicts rigid-body kinematics and Eq. (torqueSF).
                     * Reading: u_k = v_k + w_k x (r_j - r_k). */
                    double wxr[3];
                    vcross(s->omg + 3 * k, arm + 3 * m, wxr);
                    for (int a = 0; a < 3; ++a) uk[3 * m + a] = s->vel[3 * k + a] + wxr[a];
                }
                double fstar[19];
                or_cell_collide(f, s->p.tau, s->p.collision, s->p.fluid_force, ns, B, uk, arm, fstar, Fk, Mk);
                for (int m = 0; m < ns; ++m) {
                    int k = cs[c].id[m];
                    for (int a = 0; a < 3; ++a) {
#pragma omp atomic
                        s->Fh[3 * k + a] += Fk[3 * m + a];
#pragma omp atomic
                        s->Mh[3 * k + a] += Mk[3 * m + a];
                    }
                }
                /* Streaming: f_i(x + c_i, t+1) = f*_i(x, t). A link that leaves the fluid
                 * through a wall returns to x in the opposite direction, minus
                 * 2 t_i rho_w (c_i . u_w) / c_s^2 for a moving wall. Readings: rho_w is the
                 * reference density 1 (Ladd's rho_0); a link crossing walls on two axes
                 * (an edge) bounces back too and takes the velocity of the wall on the
                 * higher axis (z over y over x). */
                for (int i = 0; i < 19; ++i) {
                    int d[3] = {x + CV[i][0], y + CV[i][1], z + CV[i][2]};
                    int wall_axis = -1, wall_side = 0;
                    for (int a = 0; a < 3; ++a) {
                        if (s->periodic[a]) {
                            d[a] %= n3[a];
                            if (d[a] < 0) d[a] += n3[a];
                        } else if (d[a] < 0 || d[a] >= n3[a]) {
                            wall_axis = a;
                            wall_side = d[a] < 0 ? 0 : 1;
                        }
                    }
                    if (wall_axis < 0) {
                        long long dc = d[0] + (long long)s->nx * (d[1] + (long long)s->ny * d[2]);
                        s->fn[19 * dc + i] = fstar[i];
                    } else {
                        const double* uw = s->u_wall[wall_axis][wall_side];
                        double cu = CV[i][0] * uw[0] + CV[i][1] * uw[1] + CV[i][2] * uw[2];
                        double rho_w = 1.0;
                        s->fn[19 * c + OPP(i)] = fstar[i] - 2.0 * TW(i) * rho_w * cu / cs2;
                    }
                }
            }
    s->nsolid_overflow += over;
    double* t = s->f;
    s->f = s->fn;
    s->fn = t;
    free(cs);
}

/* ------------------------------------------------------------------------------------ */
/* DEM: integration (Sec. 2.2)                                                            */
/* ------------------------------------------------------------------------------------ */

/* Orientation as a unit quaternion q = (w, x, y, z) of the rotation that takes body
 * components to world components: that rotation's matrix has the triad d1, d2, d3 as
 * its columns (R, with the triad as rows, is its transpose). The matrix of q is the
 * textbook one, e.g. its (0,1) entry is 2(xy - wz). */
void or_triad_from_quat(const double q[4], double d[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    double m[3][3];
    m[0][0] = 1.0 - 2.0 * (y * y + z * z);
    m[0][1] = 2.0 * (x * y - w * z);
    m[0][2] = 2.0 * (x * z + w * y);
    m[1][0] = 2.0 * (x * y + w * z);
    m[1][1] = 1.0 - 2.0 * (x * x + z * z);
    m[1][2] = 2.0 * (y * z - w * x);
    m[2][0] = 2.0 * (x * z - w * y);
    m[2][1] = 2.0 * (y * z + w * x);
    m[2][2] = 1.0 - 2.0 * (x * x + y * y);
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) d[3 * i + a] = m[a][i];   /* d_i = column i */
}

/* Inverse of or_triad_from_quat (Shepperd, J. Guid. Control 1, 1978): of the four
 * quantities 4w^2, 4x^2, 4y^2, 4z^2 obtainable from the diagonal, take the largest
 * from its square root and the other three from off-diagonal sums and differences;
 * then normalise (the triad may carry rounding). */
void or_quat_from_triad(const double d[9], double q[4]) {
    double m[3][3];
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) m[a][i] = d[3 * i + a];
    const double tr = m[0][0] + m[1][1] + m[2][2];
    double w, x, y, z;
    if (tr >= m[0][0] && tr >= m[1][1] && tr >= m[2][2]) {
        w = 0.5 * sqrt(1.0 + tr);
        x = (m[2][1] - m[1][2]) / (4.0 * w);
        y = (m[0][2] - m[2][0]) / (4.0 * w);
        z = (m[1][0] - m[0][1]) / (4.0 * w);
    } else if (m[0][0] >= m[1][1] && m[0][0] >= m[2][2]) {
        x = 0.5 * sqrt(1.0 + m[0][0] - m[1][1] - m[2][2]);
        w = (m[2][1] - m[1][2]) / (4.0 * x);
        y = (m[0][1] + m[1][0]) / (4.0 * x);
        z = (m[0][2] + m[2][0]) / (4.0 * x);
    } else if (m[1][1] >= m[2][2]) {
        y = 0.5 * sqrt(1.0 - m[0][0] + m[1][1] - m[2][2]);
        w = (m[0][2] - m[2][0]) / (4.0 * y);
        x = (m[0][1] + m[1][0]) / (4.0 * y);
        z = (m[1][2] + m[2][1]) / (4.0 * y);
    } else {
        z = 0.5 * sqrt(1.0 - m[0][0] - m[1][1] + m[2][2]);
        w = (m[1][0] - m[0][1]) / (4.0 * z);
        x = (m[0][2] + m[2][0]) / (4.0 * z);
        y = (m[1][2] + m[2][1]) / (4.0 * z);
    }
    const double nq = sqrt(w * w + x * x + y * y + z * z);
    q[0] = w / nq;
    q[1] = x / nq;
    q[2] = y / nq;
    q[3] = z / nq;
}

/* Quaternion orientation update (the option in place of the triad update): the body
 * turns about the world axis w(t) by the angle |w(t)| dt, exactly,
 *   q <- (cos(|w| dt/2), sin(|w| dt/2) w/|w|) (x) q,
 * with the Hamilton product (a0, a) (x) (b0, b) = (a0 b0 - a.b, a0 b + b0 a + a x b),
 * then q is normalised and the triad rebuilt from it. The triad update of Sec. 2.2 is
 * the second-order Taylor expansion of the same rotation, so the two agree to
 * O(dt^3) per step. */
static void rotate_quat(double d[9], const double w[3], double dt) {
    double q[4], dq[4], r[4];
    or_quat_from_triad(d, q);
    const double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double c = 1.0, sn = 0.0;
    if (wn > 0.0) {
        c = cos(0.5 * dt * wn);
        sn = sin(0.5 * dt * wn) / wn;
    }
    dq[0] = c;
    for (int a = 0; a < 3; ++a) dq[1 + a] = sn * w[a];
    double ab[3];
    vcross(dq + 1, q + 1, ab);
    r[0] = dq[0] * q[0] - vdot(dq + 1, q + 1);
    for (int a = 0; a < 3; ++a) r[1 + a] = dq[0] * q[1 + a] + q[0] * dq[1 + a] + ab[a];
    const double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    for (int m = 0; m < 4; ++m) r[m] /= nr;
    or_triad_from_quat(r, d);
}

/* Predictor: Eq. (advance-r) for the position, then the orientation triad
 *   d_i* = d_i + dt w x d_i,   d_i <- d_i + dt w x (d_i + d_i*)/2,
 * re-orthonormalised (or, with orient = OR_ORIENT_QUAT, the exact rotation of
 * rotate_quat); positions wrapped into the box on periodic axes. */
static void predict(or_sim* s, double dt) {
    for (int k = 0; k < s->n; ++k) {
        double* r = s->pos + 3 * k;
        for (int a = 0; a < 3; ++a)
            r[a] = r[a] + dt * s->vel[3 * k + a] + (dt * dt / 2.0) * s->acc[3 * k + a];
        for (int a = 0; a < 3; ++a)
            if (s->periodic[a]) r[a] = r[a] - s->L[a] * floor((r[a] - s->lo[a]) / s->L[a]);
        double* d = s->triad + 9 * k;
        const double* w = s->omg + 3 * k;
        if (s->p.orient == OR_ORIENT_QUAT) {
            rotate_quat(d, w, dt);
            continue;
        }
        for (int m = 0; m < 3; ++m) {
            double* dm = d + 3 * m;
            double wxd[3], ds[3], mid[3], wxm[3];
            vcross(w, dm, wxd);
            for (int a = 0; a < 3; ++a) ds[a] = dm[a] + dt * wxd[a];
            for (int a = 0; a < 3; ++a) mid[a] = 0.5 * (dm[a] + ds[a]);
            vcross(w, mid, wxm);
            for (int a = 0; a < 3; ++a) dm[a] = dm[a] + dt * wxm[a];
        }
        orthonormalise(d);
    }
}

/* Corrector: a(t+dt) = F/m + g_b, v += dt/2 (a + a'); angular acceleration from the
 * body-frame Euler equations, Eq. (advance-omega):
 *   alpha = R^T I^-1 [ R M - (R w) x (I R w) ],  w += dt/2 (alpha + alpha').
 * R has the triad d_i as rows, so R maps world components to body components; the
 * paper's bracket is garbled, and this reading is the body-frame Euler equation with
 * the gyroscopic term evaluated at w(t). R is the triad after the predictor, i.e. the
 * orientation at which M was evaluated. g_b = g (1 - rho_f/rho_p), the analytic
 * buoyancy of Sec. 4.6. */
static void correct(or_sim* s, double dt, const double* Fh, const double* Mh) {
    for (int k = 0; k < s->n; ++k) {
        double F[3], M[3];
        for (int a = 0; a < 3; ++a) {
            F[a] = s->Fc[3 * k + a] + Fh[3 * k + a];
            M[a] = s->Mc[3 * k + a] + Mh[3 * k + a];
        }
        double an[3];
        double gfac = 1.0 - s->p.rho_f / s->rho_p[k];
        for (int a = 0; a < 3; ++a) an[a] = F[a] / s->mass[k] + s->p.gravity[a] * gfac;
        const double* d = s->triad + 9 * k;
        const double* w = s->omg + 3 * k;
        const double* I = s->inertia + 3 * k;
        double wb[3], Mb[3], Iw[3], gyr[3], ab[3], al[3];
        for (int m = 0; m < 3; ++m) {
            wb[m] = vdot(d + 3 * m, w);
            Mb[m] = vdot(d + 3 * m, M);
        }
        for (int m = 0; m < 3; ++m) Iw[m] = I[m] * wb[m];
        vcross(wb, Iw, gyr);
        for (int m = 0; m < 3; ++m) ab[m] = (Mb[m] - gyr[m]) / I[m];
        for (int a = 0; a < 3; ++a)
            al[a] = ab[0] * d[0 + a] + ab[1] * d[3 + a] + ab[2] * d[6 + a];
        for (int a = 0; a < 3; ++a) {
            s->vel[3 * k + a] += dt / 2.0 * (s->acc[3 * k + a] + an[a]);
            s->omg[3 * k + a] += dt / 2.0 * (s->alpha[3 * k + a] + al[a]);
            s->acc[3 * k + a] = an[a];
            s->alpha[3 * k + a] = al[a];
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* DEM: uniform grid / cell-linked list (Sec. 3.2.1)                                      */
/* ------------------------------------------------------------------------------------ */

/* Cell of a particle: k_a = floor((r_a - lo_a)/h_a) clamped to [0, n_a-1]. */
static unsigned cell_key(const or_sim* s, const double r[3]) {
    int k[3];
    for (int a = 0; a < 3; ++a) {
        double q = floor((r[a] - s->lo[a]) / s->gh[a]);
        int v;
        if (!(q >= 0.0)) v = 0;            /* also catches a non-finite position */
        else if (q > s->gn[a] - 1) v = s->gn[a] - 1;
        else v = (int)q;
        k[a] = v;
    }
    return (unsigned)(k[0] + s->gn[0] * (k[1] + s->gn[1] * k[2]));
}

typedef struct {
    unsigned key;
    int id;
} key_id;

static int cmp_key_id(const void* A, const void* B) {
    const key_id* a = (const key_id*)A;
    const key_id* b = (const key_id*)B;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->id < b->id ? -1 : (a->id > b->id);
}

/* Keys, then (key, id) sorted lexicographically (the grid of Sec. 3.2.1 expressed with
 * a sort, as in Table 1). */
int or_cell_keys(or_sim* s, unsigned* keys, int* sorted_ids, int grid_n[3]) {
    key_id* kv = (key_id*)xcalloc(s->n, sizeof(key_id));
    for (int k = 0; k < s->n; ++k) {
        kv[k].key = cell_key(s, s->pos + 3 * k);
        kv[k].id = k;
        if (keys) keys[k] = kv[k].key;
    }
    qsort(kv, s->n, sizeof(key_id), cmp_key_id);
    if (sorted_ids)
        for (int k = 0; k < s->n; ++k) sorted_ids[k] = kv[k].id;
    for (int a = 0; a < 3; ++a) grid_n[a] = s->gn[a];
    free(kv);
    return s->n;
}

typedef struct {
    int i, j;
} pair_ij;

static int cmp_pair(const void* A, const void* B) {
    const pair_ij* a = (const pair_ij*)A;
    const pair_ij* b = (const pair_ij*)B;
    if (a->i != b->i) return a->i < b->i ? -1 : 1;
    return a->j < b->j ? -1 : (a->j > b->j);
}

/* Candidate pairs (Sec. 3.2.1, Fig. collision-scheme): a PULL over grid cells; each
 * particle i of a cell pairs with every j > i found in the 27 neighbouring cells
 * (periodic wrap, no wrap across walls); then a lexicographic sort and unique. */
static pair_ij* candidate_pairs(const or_sim* s, int* ncand) {
    int G = s->gn[0] * s->gn[1] * s->gn[2];
    key_id* kv = (key_id*)xcalloc(s->n, sizeof(key_id));
    for (int k = 0; k < s->n; ++k) {
        kv[k].key = cell_key(s, s->pos + 3 * k);
        kv[k].id = k;
    }
    qsort(kv, s->n, sizeof(key_id), cmp_key_id);
    int* start = (int*)xcalloc(G + 1, sizeof(int));
    for (int k = 0; k < s->n; ++k) start[kv[k].key + 1]++;
    for (int g = 0; g < G; ++g) start[g + 1] += start[g];
    int cap = 64, cnt = 0;
    pair_ij* out = (pair_ij*)xcalloc(cap, sizeof(pair_ij));
    for (int g = 0; g < G; ++g) {
        int c[3] = {g % s->gn[0], (g / s->gn[0]) % s->gn[1], g / (s->gn[0] * s->gn[1])};
        for (int p = start[g]; p < start[g + 1]; ++p) {
            int i = kv[p].id;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int q[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
                        int ok = 1;
                        for (int a = 0; a < 3; ++a) {
                            if (q[a] < 0 || q[a] >= s->gn[a]) {
                                if (s->periodic[a]) q[a] = (q[a] + s->gn[a]) % s->gn[a];
                                else ok = 0;
                            }
                        }
                        if (!ok) continue;
                        int h = q[0] + s->gn[0] * (q[1] + s->gn[1] * q[2]);
                        for (int r = start[h]; r < start[h + 1]; ++r) {
                            int j = kv[r].id;
                            if (i < j) {
                                if (cnt == cap) {
                                    cap *= 2;
                                    out = (pair_ij*)realloc(out, cap * sizeof(pair_ij));
                                    if (!out) abort();
                                }
                                out[cnt].i = i;
                                out[cnt].j = j;
                                cnt++;
                            }
                        }
                    }
        }
    }
    qsort(out, cnt, sizeof(pair_ij), cmp_pair);
    int u = 0;
    for (int p = 0; p < cnt; ++p)
        if (u == 0 || out[p].i != out[u - 1].i || out[p].j != out[u - 1].j) out[u++] = out[p];
    free(kv);
    free(start);
    *ncand = u;
    return out;
}

/* ------------------------------------------------------------------------------------ */
/* Ellipsoid contact: common-normal iteration with osculating spheres (Sec. 2.1).          */
/* The paper gives the idea and cites Lambert et al.; the steps are a reading:            */
/*  (0) p_i, p_j: intersections of each surface with the centre-to-centre segment;        */
/*  (k) at p, the outward normal n and the curvature radius rho of Eq. (local-curvature)  */
/*      in body coordinates give the osculating centre o = p - rho n; the line o_i -> o_j */
/*      meets each ellipsoid at p' on the side facing the other particle. The plain       */
/*      update p <- p' oscillates and diverges for most random orientations, so each      */
/*      point moves half way, p + (p' - p)/2, and is projected back onto its surface      */
/*      along the ray from its centre. Stop when the undamped step |p' - p| of both       */
/*      points is below tol * (smallest semi-axis), after max_iter iterations, or when a  */
/*      line misses its ellipsoid (not converged).                                        */
/*  Then delta = rho_i + rho_j - |o_i - o_j|, e_n = (o_i - o_j)/|o_i - o_j|, contact     */
/*  point = midpoint of p_i, p_j.                                                         */
/* ------------------------------------------------------------------------------------ */
/* Body components of a world vector (R has the triad as rows) and back. */
static void to_body(const double R[9], const double v[3], double o[3]) {
    for (int m = 0; m < 3; ++m) o[m] = R[3 * m] * v[0] + R[3 * m + 1] * v[1] + R[3 * m + 2] * v[2];
}
static void to_world(const double R[9], const double b[3], double o[3]) {
    for (int a = 0; a < 3; ++a) o[a] = b[0] * R[a] + b[1] * R[3 + a] + b[2] * R[6 + a];
}

/* Outward unit normal, curvature radius (Eq. local-curvature) and osculating centre. */
static void osculate(const double r[3], const double R[9], const double s[3],
                     const double p[3], double n[3], double* rho, double o[3]) {
    double rel[3] = {p[0] - r[0], p[1] - r[1], p[2] - r[2]};
    double pb[3];
    to_body(R, rel, pb);
    double nb[3] = {pb[0] / (s[0] * s[0]), pb[1] / (s[1] * s[1]), pb[2] / (s[2] * s[2])};
    double nn = vnorm(nb);
    for (int m = 0; m < 3; ++m) nb[m] /= nn;
    to_world(R, nb, n);
    double a = s[0], b = s[1], c = s[2];
    *rho = b * c * pb[0] * pb[0] / (a * a * a) + a * c * pb[1] * pb[1] / (b * b * b) +
           a * b * pb[2] * pb[2] / (c * c * c);
    for (int m = 0; m < 3; ++m) o[m] = p[m] - (*rho) * n[m];
}

/* Largest root t of |body(origin + t dir - r) / s| = 1; returns 0 if the line misses. */
static int line_hit(const double r[3], const double R[9], const double s[3],
                    const double origin[3], const double dir[3], double* t) {
    double rel[3] = {origin[0] - r[0], origin[1] - r[1], origin[2] - r[2]};
    double q[3], w[3];
    to_body(R, rel, q);
    to_body(R, dir, w);
    double A = 0, B = 0, C = -1.0;
    for (int m = 0; m < 3; ++m) {
        A += (w[m] / s[m]) * (w[m] / s[m]);
        B += q[m] * w[m] / (s[m] * s[m]);
        C += (q[m] / s[m]) * (q[m] / s[m]);
    }
    double disc = B * B - A * C;
    if (disc < 0.0 || A <= 0.0) return 0;
    *t = (-B + sqrt(disc)) / A;
    return 1;
}

/* Perram-Wertheim separation certificate (Perram & Wertheim, J. Comput. Phys. 58, 409,
 * 1985). Not part of the oracle's step (the method decides ellipsoid contacts by the
 * common-normal iteration alone); it states the screening test that the CUDA contact
 * kernel runs before its iteration, so that the tests can list the pairs where the
 * screened and unscreened decisions differ. With A^-1 = R^T diag(s^2) R for each ellipsoid (R rows = body axes) and d the
 * centre difference, F(l) = l (1 - l) d^T C(l)^-1 d, C(l) = (1 - l) A_i^-1 + l A_j^-1;
 * the ellipsoids overlap if and only if max over l in [0, 1] of F is at most 1, so any l
 * with F(l) > 1 proves that they are disjoint. */
static void pw_inv_shape(const double* R, const double* s, double M[6]) {
    /* symmetric 3x3 in the order xx, yy, zz, xy, xz, yz */
    const double q0 = s[0] * s[0], q1 = s[1] * s[1], q2 = s[2] * s[2];
    M[0] = q0 * R[0] * R[0] + q1 * R[3] * R[3] + q2 * R[6] * R[6];
    M[1] = q0 * R[1] * R[1] + q1 * R[4] * R[4] + q2 * R[7] * R[7];
    M[2] = q0 * R[2] * R[2] + q1 * R[5] * R[5] + q2 * R[8] * R[8];
    M[3] = q0 * R[0] * R[1] + q1 * R[3] * R[4] + q2 * R[6] * R[7];
    M[4] = q0 * R[0] * R[2] + q1 * R[3] * R[5] + q2 * R[6] * R[8];
    M[5] = q0 * R[1] * R[2] + q1 * R[4] * R[5] + q2 * R[7] * R[8];
}

/* F(l), with C(l)^-1 d from the adjugate of the symmetric C(l). */
static double pw_F(const double Ai[6], const double Aj[6], const double d[3], double l) {
    double c[6];
    for (int k = 0; k < 6; ++k) c[k] = (1.0 - l) * Ai[k] + l * Aj[k];
    const double a00 = c[1] * c[2] - c[5] * c[5];
    const double a11 = c[0] * c[2] - c[4] * c[4];
    const double a22 = c[0] * c[1] - c[3] * c[3];
    const double a01 = c[4] * c[5] - c[3] * c[2];
    const double a02 = c[3] * c[5] - c[4] * c[1];
    const double a12 = c[3] * c[4] - c[0] * c[5];
    const double det = c[0] * a00 + c[3] * a01 + c[4] * a02;
    const double q = d[0] * (a00 * d[0] + a01 * d[1] + a02 * d[2]) +
                     d[1] * (a01 * d[0] + a11 * d[1] + a12 * d[2]) +
                     d[2] * (a02 * d[0] + a12 * d[1] + a22 * d[2]);
    return l * (1.0 - l) * q / det;
}

/* 1 if F exceeds 1 + 1e-9 at one of at most 16 values of l, taken by a golden-section
 * search for the maximum of F from the bracket [0, 1]; 0 if none does (no conclusion). */
int or_pw_separated(const double ri[3], const double Ri[9], const double si[3],
                    const double rj[3], const double Rj[9], const double sj[3]) {
    const double margin = 1.0 + 1e-9, gr = 0.6180339887498949;
    double Ai[6], Aj[6], d[3];
    pw_inv_shape(Ri, si, Ai);
    pw_inv_shape(Rj, sj, Aj);
    for (int a = 0; a < 3; ++a) d[a] = rj[a] - ri[a];
    double lo = 0.0, hi = 1.0;
    double c = hi - gr * (hi - lo), e = lo + gr * (hi - lo);
    double Fc = pw_F(Ai, Aj, d, c), Fe = pw_F(Ai, Aj, d, e);
    if (Fc > margin || Fe > margin) return 1;
    for (int k = 0; k < 14; ++k) {
        if (Fc > Fe) {
            hi = e;
            e = c;
            Fe = Fc;
            c = hi - gr * (hi - lo);
            Fc = pw_F(Ai, Aj, d, c);
            if (Fc > margin) return 1;
        } else {
            lo = c;
            c = e;
            Fc = Fe;
            e = lo + gr * (hi - lo);
            Fe = pw_F(Ai, Aj, d, e);
            if (Fe > margin) return 1;
        }
    }
    return 0;
}

int or_ellipsoid_contact(const double ri[3], const double Ri[9], const double si[3],
                         const double rj[3], const double Rj[9], const double sj[3],
                         int max_iter, double tol, double* delta, double en[3],
                         double cp[3], double* rho_i, double* rho_j, int* iters) {
    double d[3] = {rj[0] - ri[0], rj[1] - ri[1], rj[2] - ri[2]};
    double dn = vnorm(d);
    if (dn <= 0.0) return -1;
    double u[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
    double mu[3] = {-u[0], -u[1], -u[2]};
    double t;
    double pi[3], pj[3];
    if (!line_hit(ri, Ri, si, ri, u, &t)) return -1;
    for (int a = 0; a < 3; ++a) pi[a] = ri[a] + t * u[a];
    if (!line_hit(rj, Rj, sj, rj, mu, &t)) return -1;
    for (int a = 0; a < 3; ++a) pj[a] = rj[a] + t * mu[a];
    double smin = si[0];
    for (int m = 0; m < 3; ++m) {
        if (si[m] < smin) smin = si[m];
        if (sj[m] < smin) smin = sj[m];
    }
    int converged = 0, it;
    double ni[3], nj[3], oi[3], oj[3], ri_c, rj_c;
    for (it = 0; it < max_iter; ++it) {
        osculate(ri, Ri, si, pi, ni, &ri_c, oi);
        osculate(rj, Rj, sj, pj, nj, &rj_c, oj);
        double w[3] = {oj[0] - oi[0], oj[1] - oi[1], oj[2] - oi[2]};
        double wn = vnorm(w);
        if (wn <= 0.0) break;
        for (int a = 0; a < 3; ++a) w[a] /= wn;
        double mw[3] = {-w[0], -w[1], -w[2]};
        double ti, tj, npi[3], npj[3];
        if (!line_hit(ri, Ri, si, oi, w, &ti)) break;
        if (!line_hit(rj, Rj, sj, oj, mw, &tj)) break;
        for (int a = 0; a < 3; ++a) {
            npi[a] = oi[a] + ti * w[a];
            npj[a] = oj[a] + tj * mw[a];
        }
        double di[3] = {npi[0] - pi[0], npi[1] - pi[1], npi[2] - pi[2]};
        double dj[3] = {npj[0] - pj[0], npj[1] - pj[1], npj[2] - pj[2]};
        double mv = vnorm(di) > vnorm(dj) ? vnorm(di) : vnorm(dj);
        /* half step, then back onto each surface along the ray from its centre */
        double qi[3], qj[3];
        for (int a = 0; a < 3; ++a) {
            qi[a] = (pi[a] + 0.5 * di[a]) - ri[a];
            qj[a] = (pj[a] + 0.5 * dj[a]) - rj[a];
        }
        double qin = vnorm(qi), qjn = vnorm(qj);
        for (int a = 0; a < 3; ++a) {
            qi[a] /= qin;
            qj[a] /= qjn;
        }
        if (!line_hit(ri, Ri, si, ri, qi, &ti)) break;
        if (!line_hit(rj, Rj, sj, rj, qj, &tj)) break;
        for (int a = 0; a < 3; ++a) {
            pi[a] = ri[a] + ti * qi[a];
            pj[a] = rj[a] + tj * qj[a];
        }
        if (mv < tol * smin) {
            converged = 1;
            ++it;
            break;
        }
    }
    osculate(ri, Ri, si, pi, ni, &ri_c, oi);
    osculate(rj, Rj, sj, pj, nj, &rj_c, oj);
    double g[3] = {oi[0] - oj[0], oi[1] - oj[1], oi[2] - oj[2]};
    double gn = vnorm(g);
    *delta = ri_c + rj_c - gn;
    for (int a = 0; a < 3; ++a) {
        en[a] = g[a] / gn;
        cp[a] = 0.5 * (pi[a] + pj[a]);
    }
    *rho_i = ri_c;
    *rho_j = rj_c;
    *iters = it;
    return converged ? 0 : 1;
}

/* ------------------------------------------------------------------------------------ */
/* DEM: contact geometry and force (Sec. 2.1, App. A)                                     */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    double delta;     /* normal overlap, Eq. (distanceSpheres) for spheres */
    double en[3];     /* unit normal from j to i                           */
    double rci[3];    /* arm from the centre of i to the contact point      */
    double rcj[3];    /* arm from the centre of j to the contact point      */
    double Ri, Rj;    /* radii (spheres) or curvature radii (ellipsoids)    */
    int sphere;       /* both spheres: torque by the M/R form of Sec. 2.1   */
} contact_geom;

/* Sphere pair: delta = (R_i + R_j) - |r_i - r_j| (minimum image). The predicate is
 * evaluated as written: dx*dx + dy*dy + dz*dz summed left to right, then sqrt. */
static int sphere_geom(const or_sim* s, int i, int j, contact_geom* g) {
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = min_image(s, a, s->pos[3 * i + a] - s->pos[3 * j + a]);
    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double dist = sqrt(d2);
    g->delta = (s->radius[i] + s->radius[j]) - dist;
    if (!(g->delta > 0.0)) return 0;
    for (int a = 0; a < 3; ++a) g->en[a] = d[a] / dist;
    g->Ri = s->radius[i];
    g->Rj = s->radius[j];
    for (int a = 0; a < 3; ++a) {
        g->rci[a] = -g->Ri * g->en[a];
        g->rcj[a] = g->Rj * g->en[a];
    }
    g->sphere = 1;
    return 1;
}

/* Pair involving an ellipsoid: bounding-sphere test, then the common-normal iteration
 * (no other screening: the method as Sec. 2.1 states it). */
static int ellipsoid_geom(or_sim* s, int i, int j, contact_geom* g) {
    double d[3], rj_img[3];
    for (int a = 0; a < 3; ++a) {
        d[a] = min_image(s, a, s->pos[3 * i + a] - s->pos[3 * j + a]);
        rj_img[a] = s->pos[3 * i + a] - d[a];
    }
    double dist = vnorm(d);
    /* Sec. 2.1: bounding spheres (radius = largest semi-axis) select the pairs that get
     * the common-normal iteration; the iteration alone decides the contact. */
    if (!((s->bound[i] + s->bound[j]) - dist > 0.0)) return 0;
    double en[3], cp[3], rho_i, rho_j, delta;
    int iters;
    int rc = or_ellipsoid_contact(s->pos + 3 * i, s->triad + 9 * i, s->semi + 3 * i, rj_img,
                                  s->triad + 9 * j, s->semi + 3 * j, s->p.ell_max_iter,
                                  s->p.ell_tol, &delta, en, cp, &rho_i, &rho_j, &iters);
    if (rc < 0) return 0;
    if (rc > 0) s->ell_nonconverged++;
    if (!(delta > 0.0)) return 0;
    g->delta = delta;
    for (int a = 0; a < 3; ++a) {
        g->en[a] = en[a];
        g->rci[a] = cp[a] - s->pos[3 * i + a];
        g->rcj[a] = cp[a] - rj_img[a];
    }
    g->Ri = rho_i;
    g->Rj = rho_j;
    g->sphere = 0;
    return 1;
}

static int pair_geom(or_sim* s, int i, int j, contact_geom* g) {
    if (s->shape[i] == OR_SPHERE && s->shape[j] == OR_SPHERE) return sphere_geom(s, i, j, g);
    return ellipsoid_geom(s, i, j, g);
}

/* Spring-dashpot force on i (Eq. spring_dashpot_easy, Eq. fnScal), tangential history
 * (Eq. trangential-history), Coulomb limit (Eq. coulombCoeff).
 *   Rstar, mstar: Eqs. (relative_radius), (relative_mass);
 *   vi, wi, vj, wj: velocities; hist: tangential displacement (updated in place).
 * Readings where the paper is silent or garbled:
 *  - the relative surface velocity generalises Eq. (relative_velocity) to an arm:
 *    v_rel = (v_i + w_i x rc_i) - (v_j + w_j x rc_j), which is Eq. (relative_velocity)
 *    for spheres (rc_i = -R_i e_n, rc_j = R_j e_n); v_n = (v_rel . e_n) e_n, v_t = v_rel - v_n
 *    (the paper's v_n uses v_j - v_i, inconsistent in sign with v_t = v_rel - v_n);
 *  - the normal damping uses -(v_rel . e_n), equal to (v_j - v_i) . e_n for spheres;
 *  - the stored displacement is first rotated into the current tangent plane keeping
 *    its length, then incremented by v_t dt;
 *  - when |F_t| > mu |F_n| the force is scaled to the cone and the displacement reset
 *    to -(F_t + gamma_t v_t)/k_t (Cundall-Strack);
 *  - no clamp of F_n at zero.
 * Coefficients: LINEAR: k_n, k_t given; gamma = -2 beta sqrt(k m*).
 * HERTZ (App. A): k_n = 4/3 Y* sqrt(R* delta), k_t = 8 G* sqrt(R* delta),
 *   gamma_n = -2 sqrt(5/6) beta sqrt(S_n m*), S_n = 2 Y* sqrt(R* delta) (the paper's E* is
 *   read as Y*), gamma_t = -2 sqrt(5/6) beta sqrt(S_t m*), S_t = 8 G* sqrt(R* delta);
 *   beta = ln(eps)/sqrt(ln^2(eps) + pi^2). One material for every particle and wall. */
static void spring_dashpot(const or_sim* s, const contact_geom* g, double Rstar, double mstar,
                           const double vi[3], const double wi[3], const double vj[3],
                           const double wj[3], double* hist, double dt, double F[3]) {
    const double pi = 3.14159265358979323846;
    double eps = s->p.restitution;
    double beta = 0.0;
    if (eps > 0.0 && eps < 1.0) {
        double le = log(eps);
        beta = le / sqrt(le * le + pi * pi);
    } else if (eps <= 0.0) {
        beta = -1.0;
    }
    double kn, kt, gn, gt;
    if (s->p.law == OR_LAW_LINEAR) {
        kn = s->p.k_n;
        kt = s->p.k_t;
        gn = -2.0 * beta * sqrt(kn * mstar);
        gt = -2.0 * beta * sqrt(kt * mstar);
    } else {
        double E = s->p.young, nu = s->p.poisson;
        double Ystar = 1.0 / ((1.0 - nu * nu) / E + (1.0 - nu * nu) / E);
        double Gstar = 1.0 / (2.0 * (2.0 - nu) * (1.0 + nu) / E + 2.0 * (2.0 - nu) * (1.0 + nu) / E);
        double sq = sqrt(Rstar * g->delta);
        kn = 4.0 / 3.0 * Ystar * sq;
        kt = 8.0 * Gstar * sq;
        double Sn = 2.0 * Ystar * sq;
        double St = 8.0 * Gstar * sq;
        gn = -2.0 * sqrt(5.0 / 6.0) * beta * sqrt(Sn * mstar);
        gt = -2.0 * sqrt(5.0 / 6.0) * beta * sqrt(St * mstar);
    }
    double ci[3], cj[3], vrel[3];
    vcross(wi, g->rci, ci);
    vcross(wj, g->rcj, cj);
    for (int a = 0; a < 3; ++a) vrel[a] = (vi[a] + ci[a]) - (vj[a] + cj[a]);
    double vn = vdot(vrel, g->en);
    double vt[3];
    for (int a = 0; a < 3; ++a) vt[a] = vrel[a] - vn * g->en[a];
    double fn = kn * g->delta - gn * vn;
    double Fn[3];
    for (int a = 0; a < 3; ++a) Fn[a] = fn * g->en[a];
    /* tangential displacement */
    double h[3] = {hist[0], hist[1], hist[2]};
    double hn = vdot(h, g->en);
    double hp[3];
    for (int a = 0; a < 3; ++a) hp[a] = h[a] - hn * g->en[a];
    double lh = vnorm(h), lp = vnorm(hp);
    if (lp > 0.0)
        for (int a = 0; a < 3; ++a) hp[a] *= lh / lp;
    for (int a = 0; a < 3; ++a) h[a] = hp[a] + vt[a] * dt;
    double Ft[3];
    for (int a = 0; a < 3; ++a) Ft[a] = -kt * h[a] - gt * vt[a];
    double lft = vnorm(Ft), lfn = fabs(fn);
    if (lft > s->p.friction * lfn) {
        double sc = lft > 0.0 ? s->p.friction * lfn / lft : 0.0;
        for (int a = 0; a < 3; ++a) Ft[a] *= sc;
        if (kt > 0.0)
            for (int a = 0; a < 3; ++a) h[a] = -(Ft[a] + gt * vt[a]) / kt;
    }
    for (int a = 0; a < 3; ++a) {
        hist[a] = h[a];
        F[a] = Fn[a] + Ft[a];
    }
}

/* Tangential part of F with respect to e_n (used by the sphere torque form). */
static void tangential_part(const double F[3], const double en[3], double Ft[3]) {
    double fn = vdot(F, en);
    for (int a = 0; a < 3; ++a) Ft[a] = F[a] - fn * en[a];
}

static double relative(double a, double b) { return 1.0 / (1.0 / a + 1.0 / b); }

/* Particle-wall contact (Sec. 2.1, last paragraph): the wall is a static infinite plane
 * at the halfway bounce-back position with a surface velocity; infinite mass and radius
 * (R* = R_i, m* = m_i). face = 2*axis + side. Returns 1 on contact. */
static int wall_geom(const or_sim* s, int k, int face, contact_geom* g) {
    int a = face / 2, side = face % 2;
    double nrm[3] = {0, 0, 0};
    nrm[a] = side == 0 ? 1.0 : -1.0;   /* inward normal, from the wall to the particle */
    const double* r = s->pos + 3 * k;
    if (s->shape[k] == OR_SPHERE) {
        double dist = side == 0 ? r[a] - s->lo[a] : s->hi[a] - r[a];
        g->delta = s->radius[k] - dist;
        if (!(g->delta > 0.0)) return 0;
        for (int b = 0; b < 3; ++b) {
            g->en[b] = nrm[b];
            g->rci[b] = -s->radius[k] * nrm[b];
            g->rcj[b] = 0.0;
        }
        g->Ri = s->radius[k];
        g->sphere = 1;
        return 1;
    }
    /* Ellipsoid: support point towards the wall, p = r - E n / sqrt(n.E n) with
     * E = R^T diag(s^2) R, computed in the body frame (closed form). */
    const double* R = s->triad + 9 * k;
    const double* sa = s->semi + 3 * k;
    double nb[3], pb[3], p[3], pw[3];
    to_body(R, nrm, nb);
    double den = sqrt(sa[0] * sa[0] * nb[0] * nb[0] + sa[1] * sa[1] * nb[1] * nb[1] +
                      sa[2] * sa[2] * nb[2] * nb[2]);
    for (int m = 0; m < 3; ++m) pb[m] = -sa[m] * sa[m] * nb[m] / den;
    to_world(R, pb, pw);
    for (int b = 0; b < 3; ++b) p[b] = r[b] + pw[b];
    double sd = side == 0 ? p[a] - s->lo[a] : s->hi[a] - p[a];
    g->delta = -sd;
    if (!(g->delta > 0.0)) return 0;
    double n_[3], rho, o[3];
    osculate(r, R, sa, p, n_, &rho, o);
    for (int b = 0; b < 3; ++b) {
        g->en[b] = nrm[b];
        g->rci[b] = (p[b] + 0.5 * g->delta * nrm[b]) - r[b];
        g->rcj[b] = 0.0;
    }
    g->Ri = rho;
    g->sphere = 0;
    return 1;
}

/* Table 1 "Compute DEM forces" and "Reduce DEM forces" at the current state:
 * contact list (candidate pairs filtered by overlap, sorted by (i,j)), tangential
 * history looked up by binary search in the previous sorted list (Sec. 3.2.2), the
 * force stored once per pair and the torque per member, then per-particle sums over
 * pairs where the particle is the left member and then the right member, and walls. */
void or_contact_forces(or_sim* s, double dt) {
    int ncand;
    pair_ij* cand = candidate_pairs(s, &ncand);
    int* nci = (int*)xcalloc(ncand, sizeof(int));
    int* ncj = (int*)xcalloc(ncand, sizeof(int));
    double* nh = (double*)xcalloc(3 * (size_t)ncand, sizeof(double));
    double* PF = (double*)xcalloc(3 * (size_t)ncand, sizeof(double));
    double* PMi = (double*)xcalloc(3 * (size_t)ncand, sizeof(double));
    double* PMj = (double*)xcalloc(3 * (size_t)ncand, sizeof(double));
    int nc = 0;
    for (int p = 0; p < ncand; ++p) {
        int i = cand[p].i, j = cand[p].j;
        contact_geom g;
        if (!pair_geom(s, i, j, &g)) continue;
        /* history: binary search in the previous (sorted) contact list */
        double hist[3] = {0, 0, 0};
        int lo = 0, hi = s->ncont - 1;
        while (lo <= hi) {
            int mid = (lo + hi) / 2;
            int ci = s->ci[mid], cj = s->cj[mid];
            if (ci == i && cj == j) {
                for (int a = 0; a < 3; ++a) hist[a] = s->chist[3 * mid + a];
                break;
            }
            if (ci < i || (ci == i && cj < j)) lo = mid + 1;
            else hi = mid - 1;
        }
        double Rstar = relative(g.Ri, g.Rj);
        double mstar = relative(s->mass[i], s->mass[j]);
        double F[3];
        spring_dashpot(s, &g, Rstar, mstar, s->vel + 3 * i, s->omg + 3 * i, s->vel + 3 * j,
                       s->omg + 3 * j, hist, dt, F);
        nci[nc] = i;
        ncj[nc] = j;
        for (int a = 0; a < 3; ++a) {
            nh[3 * nc + a] = hist[a];
            PF[3 * nc + a] = F[a];
        }
        if (g.sphere) {
            /* Sec. 2.1: M_ij = -R_i e_n x F_t; M/R is the same for both members. */
            double Ft[3], mr[3];
            tangential_part(F, g.en, Ft);
            vcross(g.en, Ft, mr);
            for (int a = 0; a < 3; ++a) {
                PMi[3 * nc + a] = -g.Ri * mr[a];
                PMj[3 * nc + a] = -g.Rj * mr[a];
            }
        } else {
            /* Eq. (torque): M = rc x F, with -F acting on j. */
            double mi[3], mj[3], mF[3] = {-F[0], -F[1], -F[2]};
            vcross(g.rci, F, mi);
            vcross(g.rcj, mF, mj);
            for (int a = 0; a < 3; ++a) {
                PMi[3 * nc + a] = mi[a];
                PMj[3 * nc + a] = mj[a];
            }
        }
        nc++;
    }
    /* reductions: left members (pairs already sorted by i), then right members */
    for (int k = 0; k < s->n; ++k)
        for (int a = 0; a < 3; ++a) s->Fc[3 * k + a] = s->Mc[3 * k + a] = 0.0;
    for (int p = 0; p < nc; ++p)
        for (int a = 0; a < 3; ++a) {
            s->Fc[3 * nci[p] + a] += PF[3 * p + a];
            s->Mc[3 * nci[p] + a] += PMi[3 * p + a];
        }
    for (int p = 0; p < nc; ++p)
        for (int a = 0; a < 3; ++a) {
            s->Fc[3 * ncj[p] + a] -= PF[3 * p + a];
            s->Mc[3 * ncj[p] + a] += PMj[3 * p + a];
        }
    /* walls */
    for (int k = 0; k < s->n; ++k)
        for (int face = 0; face < 6; ++face) {
            int a = face / 2;
            double* wh = s->whist + 18 * k + 3 * face;
            contact_geom g;
            if (s->periodic[a] || !wall_geom(s, k, face, &g)) {
                wh[0] = wh[1] = wh[2] = 0.0;
                continue;
            }
            const double* uw = s->u_wall[a][face % 2];
            double zero[3] = {0, 0, 0}, F[3];
            spring_dashpot(s, &g, g.Ri, s->mass[k], s->vel + 3 * k, s->omg + 3 * k, uw, zero,
                           wh, dt, F);
            double M[3];
            if (g.sphere) {
                double Ft[3], mr[3];
                tangential_part(F, g.en, Ft);
                vcross(g.en, Ft, mr);
                for (int b = 0; b < 3; ++b) M[b] = -g.Ri * mr[b];
            } else {
                vcross(g.rci, F, M);
            }
            for (int b = 0; b < 3; ++b) {
                s->Fc[3 * k + b] += F[b];
                s->Mc[3 * k + b] += M[b];
            }
        }
    /* the new list becomes the previous list */
    if (nc > s->contcap) {
        s->contcap = nc;
        s->ci = (int*)realloc(s->ci, nc * sizeof(int));
        s->cj = (int*)realloc(s->cj, nc * sizeof(int));
        s->chist = (double*)realloc(s->chist, 3 * (size_t)nc * sizeof(double));
        if (!s->ci || !s->cj || !s->chist) abort();
    }
    for (int p = 0; p < nc; ++p) {
        s->ci[p] = nci[p];
        s->cj[p] = ncj[p];
        for (int a = 0; a < 3; ++a) s->chist[3 * p + a] = nh[3 * p + a];
    }
    s->ncont = nc;
    free(cand); free(nci); free(ncj); free(nh); free(PF); free(PMi); free(PMj);
}

/* Current contact set as keys (i << 32 | j), sorted; without touching the history. */
int or_contacts(or_sim* s, long long* pair_keys, int cap) {
    int ncand;
    pair_ij* cand = candidate_pairs(s, &ncand);
    int nc = 0;
    for (int p = 0; p < ncand; ++p) {
        contact_geom g;
        long long save = s->ell_nonconverged;
        int hit = pair_geom(s, cand[p].i, cand[p].j, &g);
        s->ell_nonconverged = save;
        if (!hit) continue;
        if (nc < cap) pair_keys[nc] = ((long long)cand[p].i << 32) | (long long)cand[p].j;
        nc++;
    }
    free(cand);
    return nc;
}

/* ------------------------------------------------------------------------------------ */
/* The coupled time step, in the order of the flowchart of Sec. 3.2:                      */
/*  per DEM substep: update positions; grid; collision list; pair forces and tangential   */
/*  history; reduction. Then the PSM fluid update at the current particle state, the     */
/*  reduction of the fluid forces, and the particle velocity update.                      */
/* With n_sub > 1 (Sec. 2.3, last paragraph) the paper does not say how the fluid force  */
/* enters the intermediate substeps; reading: substeps 1..n_sub-1 complete their          */
/* velocity update with the hydrodynamic force of the previous fluid step held constant.  */
/* A DEM-only simulation (no lattice) runs every substep with a zero fluid force.         */
/* ------------------------------------------------------------------------------------ */
void or_step(or_sim* s, int nsteps) {
    int nsub = s->p.n_sub > 0 ? s->p.n_sub : 1;
    double dt = 1.0 / nsub;
    for (int st = 0; st < nsteps; ++st) {
        for (int sub = 1; sub <= nsub && s->n > 0; ++sub) {
            predict(s, dt);
            or_contact_forces(s, dt);
            if (sub < nsub || s->ncell == 0) correct(s, dt, s->Fh_prev, s->Mh_prev);
        }
        if (s->ncell > 0) {
            or_lbm_psm_step(s);
            correct(s, dt, s->Fh, s->Mh);
            memcpy(s->Fh_prev, s->Fh, sizeof(double) * 3 * s->n);
            memcpy(s->Mh_prev, s->Mh, sizeof(double) * 3 * s->n);
        }
        s->steps++;
    }
}
