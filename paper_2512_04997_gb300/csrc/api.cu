// api.cu -- C ABI of the LEDDS GB300 library (declared in include/ledds.h).
//
// Host-side orchestration: workspace layout (the library allocates no device memory),
// parameter validation, particle upload, and the coupled step of the flowchart of
// Sec. 3.2 enqueued as kernels and replayed as CUDA graphs (one graph per starting
// buffer parity for one step and for two steps, so buffers return to their roles).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace ledds {
cudaError_t launch_init(const LbmArgs&, int, const float*, const float*, const float*, cudaStream_t);
cudaError_t launch_read(const LbmArgs&, int, float*, float*, float*, int, cudaStream_t);
cudaError_t launch_rebase(const LbmArgs&, int, const float (*)[2][3], cudaStream_t);
cudaError_t launch_bin(const LbmArgs&, int, int*, int*, cudaStream_t);
cudaError_t launch_psm(const LbmArgs&, const PsmMaps*, int, cudaStream_t);
cudaError_t launch_voxelize(const LbmArgs&, float*, int*, int*, cudaStream_t);
cudaError_t launch_rebuild(const DemArgs&, int, int, int, uint32_t*, cudaStream_t, int*);
cudaError_t launch_predict_first(const DemArgs&, cudaStream_t);
cudaError_t launch_substep(const DemArgs&, int, int, int, int, int*, cudaStream_t);
cudaError_t launch_final(const DemArgs&, int, int, cudaStream_t);
cudaError_t launch_pairs(const DemArgs&, int, uint32_t*, uint32_t*, uint32_t*, unsigned long long*,
                         int, cudaStream_t);
cudaError_t launch_scan(const uint32_t*, int, uint32_t*, uint32_t*, cudaStream_t);
cudaError_t launch_psm_batch(const BatchChunk&, int*, int, int, bool, cudaStream_t);
cudaError_t launch_bin_batch(const LbmArgs*, const int*, int, cudaStream_t);
cudaError_t launch_dem_batch(const DemArgs*, const int*, int, int, cudaStream_t);
cudaError_t launch_final_batch(const DemArgs*, int, cudaStream_t);
int psm_batch_ctas_per_sm();
}  // namespace ledds

using namespace ledds;

static const double kPi = 3.14159265358979323846;
enum { NSTAGE = 5 };

struct ledds_sim_s {
    ledds_dims d;
    ledds_params p;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    // The neighbour rebuild for the next step runs on a side stream beside the fluid step
    // (it needs only the positions after the last substep); lists_ready: the current step's
    // candidate lists were built that way, at the current positions.
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    bool lists_ready = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    // lattice
    bool lattice = false;
    long long N = 0;
    int ntx = 0, nty = 0, ntz = 0, ntiles = 0;
    int tz = TILE_Z;          // tile depth (planes per tile)
    void* pop[2] = {nullptr, nullptr};
    PsmMaps maps[2];          // tensor maps of pop[0], pop[1] (staged PSM route)
    bool staged = false;      // the PSM kernel takes the staged route
    int* tile_count = nullptr;
    int* tile_ids = nullptr;
    int tile_cap = 0;
    // particles
    DevParticles P{};
    int ccap = 0;
    double lo[3], hi[3], L[3];
    int gn[3] = {1, 1, 1};
    double gh[3] = {1, 1, 1};
    int G = 1;
    uint32_t *keys = nullptr, *cell_count = nullptr, *cell_start = nullptr, *scan_partial = nullptr;
    uint32_t *pair_cnt = nullptr, *pair_off = nullptr;
    uint32_t* cp_list = nullptr;  // canonical pair list (pair-once evaluation)
    double* cp_res = nullptr;     // per-pair force and torques
    long long cp_stride = 0;
    int *rank = nullptr, *sorted = nullptr, *sorted_tmp = nullptr, *seg_big = nullptr;
    int* cand[2] = {nullptr, nullptr};
    int* ncand[2] = {nullptr, nullptr};
    double* hist[2] = {nullptr, nullptr};
    double* whist = nullptr;
    DevStatus* status = nullptr;
    int sms = 1;             // multiprocessors of the device (launch shapes)
    double max_bound = 0.0;  // largest bounding radius of the current particles
    int any_ellipsoid = 0;   // some current particle is an ellipsoid
    // state
    double uw[3][2][3];
    int parity = 0;          // pop[parity], cand[parity] hold the current data
    long long steps = 0;
    // graphs
    cudaGraphExec_t g1[2] = {nullptr, nullptr}, g2[2] = {nullptr, nullptr};
    cudaGraphExec_t grb[2] = {nullptr, nullptr};  // the leading list rebuild, per parity
    int launches_per_step = 0;
    // profiling
    bool profiling = false;
    cudaEvent_t ev[NSTAGE + 1];
    bool ev_made = false;
    double prof_ms[NSTAGE];
    long long prof_steps = 0, prof_launches = 0;
    // batch membership
    bool in_batch = false;
    long long version = 0;   // bumped by every change that invalidates captured graphs
};

// ------------------------------------------------------------------------------------
// Workspace layout
// ------------------------------------------------------------------------------------
struct Carver {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

static int check_args(const ledds_dims* d, const ledds_params* p) {
    if (!d || !p) return LEDDS_ERR_INVALID_ARG;
    if (d->nx < 0 || d->ny < 0 || d->nz < 0) return LEDDS_ERR_INVALID_ARG;
    bool lat = d->nx > 0 || d->ny > 0 || d->nz > 0;
    if (lat && (d->nx <= 0 || d->ny <= 0 || d->nz <= 0)) return LEDDS_ERR_INVALID_ARG;
    // node indices are 32-bit (population offsets become 64-bit beyond 19 N = 2^31)
    if (lat && (double)d->nx * d->ny * d->nz >= 2147483647.0) return LEDDS_ERR_INVALID_ARG;
    if (!lat && d->max_particles <= 0) return LEDDS_ERR_INVALID_ARG;
    if (d->max_particles < 0) return LEDDS_ERR_INVALID_ARG;
    if (!(p->tau > 0.5)) return LEDDS_ERR_INVALID_ARG;
    if (p->storage < 0 || p->storage > 2) return LEDDS_ERR_INVALID_ARG;
    if (p->voxel < 0 || p->voxel > 1) return LEDDS_ERR_INVALID_ARG;
    if (p->subdiv_n < 1 || p->subdiv_n > 16) return LEDDS_ERR_INVALID_ARG;
    if (p->law < 0 || p->law > 1) return LEDDS_ERR_INVALID_ARG;
    if (p->n_sub < 1) return LEDDS_ERR_INVALID_ARG;
    if (p->storage_scale_log2 < -30 || p->storage_scale_log2 > 30) return LEDDS_ERR_INVALID_ARG;
    if (d->cand_cap < 0 || d->cand_cap > MAX_CAND_CAP) return LEDDS_ERR_INVALID_ARG;
    if (d->tile_cap < 0 || d->tile_cap > MAX_TILE_CAP) return LEDDS_ERR_INVALID_ARG;
    if (d->max_particles > 0 && !(p->dem_h > 0.0)) return LEDDS_ERR_INVALID_ARG;
    if (p->skin < 0.0) return LEDDS_ERR_INVALID_ARG;
    if (p->force_fp32 < 0 || p->force_fp32 > 1) return LEDDS_ERR_INVALID_ARG;
    if (p->collision < 0 || p->collision > 1) return LEDDS_ERR_INVALID_ARG;
    if (p->orient < 0 || p->orient > 1) return LEDDS_ERR_INVALID_ARG;
    if (p->pattern < 0 || p->pattern > 1) return LEDDS_ERR_INVALID_ARG;
    if (p->index64 < 0 || p->index64 > 1) return LEDDS_ERR_INVALID_ARG;
    if (p->psm_route < 0 || p->psm_route > 2) return LEDDS_ERR_INVALID_ARG;
    if (p->ell_screen < 0 || p->ell_screen > 1) return LEDDS_ERR_INVALID_ARG;
    if (!lat) {
        for (int a = 0; a < 3; ++a)
            if (!(d->box_hi[a] > d->box_lo[a])) return LEDDS_ERR_INVALID_ARG;
    }
    return LEDDS_OK;
}

static void domain(const ledds_dims* d, double lo[3], double hi[3], double L[3]) {
    bool lat = d->nx > 0;
    int n3[3] = {d->nx, d->ny, d->nz};
    for (int a = 0; a < 3; ++a) {
        lo[a] = lat ? -0.5 : d->box_lo[a];
        hi[a] = lat ? n3[a] - 0.5 : d->box_hi[a];
        L[a] = hi[a] - lo[a];
    }
}

static void grid_of(const ledds_dims* d, const ledds_params* p, int gn[3], double gh[3], int* G) {
    double lo[3], hi[3], L[3];
    domain(d, lo, hi, L);
    *G = 1;
    for (int a = 0; a < 3; ++a) {
        int g = p->dem_h > 0 ? (int)floor(L[a] / p->dem_h) : 1;
        if (g < 1) g = 1;
        gn[a] = g;
        gh[a] = L[a] / g;
        *G *= g;
    }
}

// Lays out every device array; with base == nullptr only computes the size.
static size_t layout(ledds_sim_s* s, const ledds_dims* d, const ledds_params* p, char* base) {
    Carver c{base};
    long long N = (long long)d->nx * d->ny * d->nz;
    size_t sb = storage_bytes(p->storage);
    int ntx = (d->nx + TILE_X - 1) / TILE_X, nty = (d->ny + TILE_Y - 1) / TILE_Y,
        ntz = (d->nz + TILE_Z - 1) / TILE_Z;
    int ntiles = N > 0 ? ntx * nty * ntz : 0;
    // tile lists are sized for the smallest tile depth (a batch may choose it)
    int ntiles_alloc = N > 0 ? ntx * nty * ((d->nz + TILE_Z_MIN - 1) / TILE_Z_MIN) : 0;
    int tcap = d->tile_cap > 0 ? d->tile_cap : 64;
    int cap = d->max_particles > 0 ? d->max_particles : 0;
    int ccap = d->cand_cap > 0 ? d->cand_cap : 32;
    int gn[3];
    double gh[3];
    int G;
    grid_of(d, p, gn, gh, &G);
    int capc = cap > 0 ? cap : 1;
    void* pop0 = c.take<char>((size_t)N * 19 * sb);
    // the AA pattern steps in place: one population array
    void* pop1 = p->pattern == LEDDS_PATTERN_AA ? pop0 : c.take<char>((size_t)N * 19 * sb);
    int* tcount = c.take<int>((size_t)(ntiles_alloc > 0 ? ntiles_alloc : 1));
    int* tids = c.take<int>((size_t)(ntiles_alloc > 0 ? ntiles_alloc : 1) * tcap);
    double* st0 = c.take<double>(18 * (size_t)capc);
    double* st1 = c.take<double>(18 * (size_t)capc);
    double* acc = c.take<double>(3 * (size_t)capc);
    double* alpha = c.take<double>(3 * (size_t)capc);
    double* Fc = c.take<double>(3 * (size_t)capc);
    double* Mc = c.take<double>(3 * (size_t)capc);
    double* Fh = c.take<double>(6 * (size_t)capc);  // Fh then Mh, contiguous
    double* Fhp = c.take<double>(6 * (size_t)capc);
    double* pb = c.take<double>(3 * (size_t)capc);
    double* radius = c.take<double>((size_t)capc);
    double* semi = c.take<double>(3 * (size_t)capc);
    double* bound = c.take<double>((size_t)capc);
    double* mass = c.take<double>((size_t)capc);
    double* inertia = c.take<double>(3 * (size_t)capc);
    double* gfac = c.take<double>((size_t)capc);
    int* shape = c.take<int>((size_t)capc);
    uint32_t* keys = c.take<uint32_t>((size_t)capc);
    int* rank = c.take<int>((size_t)capc);
    int* sorted = c.take<int>((size_t)capc);
    int* sorted_tmp = c.take<int>((size_t)capc);
    int* seg_big = c.take<int>((size_t)capc / 32 + 2);
    uint32_t* ccount = c.take<uint32_t>((size_t)G + 1);
    uint32_t* cstart = c.take<uint32_t>((size_t)G + 1);
    uint32_t* partial = c.take<uint32_t>(4096);
    uint32_t* pcnt = c.take<uint32_t>((size_t)capc);
    uint32_t* poff = c.take<uint32_t>((size_t)capc + 1);
    int* cand0 = c.take<int>((size_t)capc * ccap);
    int* cand1 = c.take<int>((size_t)capc * ccap);
    int* nc0 = c.take<int>((size_t)capc);
    int* nc1 = c.take<int>((size_t)capc);
    double* h0 = c.take<double>((size_t)capc * ccap * 3);
    double* h1 = c.take<double>((size_t)capc * ccap * 3);
    double* wh = c.take<double>((size_t)capc * 18);
    uint32_t* cplist = c.take<uint32_t>((size_t)capc * ccap);
    double* cpres = c.take<double>((size_t)capc * ccap * 9);
    DevStatus* status = c.take<DevStatus>(1);
    size_t total = c.off + 256;
    if (s && base) {
        s->N = N;
        s->lattice = N > 0;
        s->ntx = ntx;
        s->nty = nty;
        s->ntz = ntz;
        s->ntiles = ntiles;
        s->tz = TILE_Z;
        s->tile_cap = tcap;
        s->pop[0] = pop0;
        s->pop[1] = pop1;
        // route 0 (automatic): staged for FP32, where it is faster; the 16-bit kernels are
        // bound by instruction issue and the per-thread loads are faster for them
        const bool want_staged = p->psm_route == 2 || (p->psm_route == 0 && p->storage == LEDDS_STORE_F32);
        s->staged = N > 0 && want_staged &&
                    psm_make_maps(pop0, p->storage, d->nx, d->ny, d->nz, &s->maps[0]) &&
                    psm_make_maps(pop1, p->storage, d->nx, d->ny, d->nz, &s->maps[1]);
        s->tile_count = tcount;
        s->tile_ids = tids;
        s->ccap = ccap;
        DevParticles& P = s->P;
        P.n = 0;
        P.cap = capc;
        P.st[0] = st0;
        P.st[1] = st1;
        P.acc = acc;
        P.alpha = alpha;
        P.Fc = Fc;
        P.Mc = Mc;
        P.Fh = Fh;
        P.Mh = Fh + 3 * (size_t)capc;
        P.Fhp = Fhp;
        P.Mhp = Fhp + 3 * (size_t)capc;
        P.pos_build = pb;
        P.radius = radius;
        P.semi = semi;
        P.bound = bound;
        P.mass = mass;
        P.inertia = inertia;
        P.gfac = gfac;
        P.shape = shape;
        s->keys = keys;
        s->rank = rank;
        s->sorted = sorted;
        s->sorted_tmp = sorted_tmp;
        s->seg_big = seg_big;
        s->cell_count = ccount;
        s->cell_start = cstart;
        s->scan_partial = partial;
        s->pair_cnt = pcnt;
        s->pair_off = poff;
        s->cand[0] = cand0;
        s->cand[1] = cand1;
        s->ncand[0] = nc0;
        s->ncand[1] = nc1;
        s->hist[0] = h0;
        s->hist[1] = h1;
        s->whist = wh;
        s->cp_list = cplist;
        s->cp_res = cpres;
        s->cp_stride = (long long)capc * ccap;
        s->status = status;
        for (int a = 0; a < 3; ++a) {
            s->gn[a] = gn[a];
            s->gh[a] = gh[a];
        }
        s->G = G;
    }
    return total;
}

static LbmArgs lbm_args(const ledds_sim_s* s, int in, int out, int pst) {
    LbmArgs a{};
    a.nx = s->d.nx;
    a.ny = s->d.ny;
    a.nz = s->d.nz;
    a.N = s->N;
    for (int q = 0; q < 3; ++q) a.per[q] = s->d.periodic[q];
    for (int q = 0; q < 3; ++q)
        for (int e = 0; e < 2; ++e)
            for (int c = 0; c < 3; ++c) a.uw[q][e][c] = (float)s->uw[q][e][c];
    a.tau = (float)s->p.tau;
    a.omega = (float)(1.0 / s->p.tau);
    for (int q = 0; q < 3; ++q) a.F[q] = (float)s->p.fluid_force[q];
    a.has_force = (s->p.fluid_force[0] != 0 || s->p.fluid_force[1] != 0 || s->p.fluid_force[2] != 0);
    a.guo_pref = (float)(1.0 - 0.5 / s->p.tau);
    a.trt = s->p.collision == LEDDS_COLLIDE_TRT;
    {
        const double wp = 1.0 / s->p.tau;
        const double wm = a.trt ? 8.0 * (2.0 - wp) / (8.0 - wp) : wp;  // Eq. (TRT) rate relation
        a.omega_m = (float)wm;
        a.guo_pref_m = (float)(1.0 - 0.5 * wm);
    }
    double sc = s->p.storage == LEDDS_STORE_F16 ? ldexp(1.0, s->p.storage_scale_log2) : 1.0;
    a.scale = (float)sc;
    a.inv_scale = (float)(1.0 / sc);
    a.pop_in = s->pop[in];
    a.pop_out = s->pop[out];
    // AA: parity 0 holds the pre-collision f (the step from it collides in place), parity 1
    // the post-collision f*_i in slot opp(i) (the step from it streams); the two pointers
    // are the same array
    a.aa = s->p.pattern != LEDDS_PATTERN_AA ? PSM_AB : (in == 0 ? PSM_AA_EVEN : PSM_AA_ODD);
    // 64-bit population offsets when 19 N elements pass the 32-bit range (or if requested)
    a.w64 = s->p.index64 || 19LL * s->N >= 2147483647LL;
    for (int i = 0; i < 19; ++i) {
        a.pN[i] = a.w64 ? 0 : (int)(i * s->N);
        a.off[i] = CX(i) + s->d.nx * (CY(i) + s->d.ny * CZ(i));
        if (a.off[i] & 1) a.off_odd |= 1u << i;
    }
    a.nx_even = (s->d.nx % 2) == 0;
    {
        // Cached centres are minimum-imaged against the tile origin; a node offset can
        // still need a wrap only if the box is narrower than the reach of a particle
        // from a tile (both sides) plus the tile itself.
        const int n3[3] = {s->d.nx, s->d.ny, s->d.nz};
        const int T[3] = {TILE_X, TILE_Y, s->tz};
        for (int q = 0; q < 3; ++q)
            a.mi[q] = s->d.periodic[q] && (double)n3[q] < 2.0 * (s->max_bound + 2.0 + T[q]) + 2.0;
    }
    a.ntx = s->ntx;
    a.nty = s->nty;
    a.ntz = s->ntz;
    a.tz = s->tz;
    // fewer tiles than two waves of CTAs: split each tile's planes over four CTAs
    a.zsplit = s->ntiles < 2 * s->sms ? 4 : 1;
    a.tile_cap = s->tile_cap;
    a.tile_count = s->tile_count;
    a.tile_ids = s->tile_ids;
    a.st = s->P.st[pst];
    a.pcap = s->P.cap;
    a.radius = s->P.radius;
    a.semi = s->P.semi;
    a.bound = s->P.bound;
    a.shape = s->P.shape;
    a.Fh = s->P.Fh;
    a.Mh = s->P.Mh;
    a.voxel = s->p.voxel;
    a.subdiv_any = s->p.voxel == LEDDS_VOXEL_SUBDIV || s->any_ellipsoid;
    a.subdiv_n = s->p.subdiv_n;
    a.Rc = (float)cbrt(3.0 / (4.0 * kPi));
    a.inv2Rc = (float)(1.0 / (2.0 * cbrt(3.0 / (4.0 * kPi))));
    a.status = s->status;
    return a;
}

static DemArgs dem_args(const ledds_sim_s* s) {
    DemArgs A{};
    A.P = s->P;
    for (int a = 0; a < 3; ++a) {
        A.lo[a] = s->lo[a];
        A.hi[a] = s->hi[a];
        A.L[a] = s->L[a];
        A.per[a] = s->d.periodic[a];
        A.gn[a] = s->gn[a];
        A.gh[a] = s->gh[a];
        A.gravity[a] = s->p.gravity[a];
    }
    memcpy(A.uw, s->uw, sizeof(A.uw));
    A.G = s->G;
    A.dt = 1.0 / s->p.n_sub;
    A.n_sub = s->p.n_sub;
    A.law = s->p.law;
    A.k_n = s->p.k_n;
    A.k_t = s->p.k_t;
    double eps = s->p.restitution;
    double beta = 0.0;
    if (eps > 0.0 && eps < 1.0) {
        double le = log(eps);
        beta = le / sqrt(le * le + kPi * kPi);
    } else if (eps <= 0.0) {
        beta = -1.0;
    }
    A.beta = beta;
    double E = s->p.young, nu = s->p.poisson;
    A.Ystar = 1.0 / ((1.0 - nu * nu) / E + (1.0 - nu * nu) / E);
    A.Gstar = 1.0 / (2.0 * (2.0 - nu) * (1.0 + nu) / E + 2.0 * (2.0 - nu) * (1.0 + nu) / E);
    A.mu = s->p.friction;
    A.skin = s->p.skin;
    A.ell_max_iter = s->p.ell_max_iter;
    A.ell_tol = s->p.ell_tol;
    A.ell_screen = s->p.ell_screen;
    A.force_f32 = s->p.force_fp32;
    A.quat = s->p.orient == LEDDS_ORIENT_QUAT;
    A.pair_once = s->any_ellipsoid;
    A.cp_cnt = s->pair_cnt;
    A.cp_off = s->pair_off;
    A.cp_list = s->cp_list;
    A.cp_res = s->cp_res;
    A.cp_stride = s->cp_stride;
    A.ccap = s->ccap;
    A.keys = s->keys;
    A.rank = s->rank;
    A.sorted = s->sorted;
    A.sorted_tmp = s->sorted_tmp;
    A.seg_big = s->seg_big;
    A.cell_count = s->cell_count;
    A.cell_start = s->cell_start;
    for (int b = 0; b < 2; ++b) {
        A.cand[b] = s->cand[b];
        A.ncand[b] = s->ncand[b];
        A.hist[b] = s->hist[b];
    }
    A.whist = s->whist;
    A.status = s->status;
    return A;
}

static void drop_graphs(ledds_sim_s* s) {
    s->version++;
    for (int q = 0; q < 2; ++q) {
        if (s->g1[q]) cudaGraphExecDestroy(s->g1[q]);
        if (s->g2[q]) cudaGraphExecDestroy(s->g2[q]);
        if (s->grb[q]) cudaGraphExecDestroy(s->grb[q]);
        s->g1[q] = s->g2[q] = s->grb[q] = nullptr;
    }
}

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

// The coupled step, flowchart order of Sec. 3.2, starting from buffer parity p.
// ev (optional) receives NSTAGE+1 events bracketing the stages.
static cudaError_t enqueue_step(ledds_sim_s* s, int p, cudaStream_t st, int* launches,
                                cudaEvent_t* ev) {
    const int n = s->P.n;
    const int nsub = s->p.n_sub;
    const int last = (nsub - 1) & 1;
    DemArgs A = dem_args(s);
    // With a lattice (and not profiling), the rebuild for the next step runs beside the
    // binning and the PSM kernel; this step's lists then come from the previous step.
    const bool overlap = s->lattice && n > 0 && !ev;
    if (ev) CK(cudaEventRecord(ev[0], st));
    if (n > 0 && !overlap) {
        // particle/grid stage: neighbour rebuild (keys, counting sort, candidates)
        CK(launch_rebuild(A, p, p ^ 1, 0, s->scan_partial, st, launches));
    }
    if (ev) CK(cudaEventRecord(ev[1], st));
    if (n > 0) {
        CK(launch_predict_first(A, st));
        *launches += 1;
        for (int sub = 1; sub < nsub; ++sub)
            CK(launch_substep(A, (sub - 1) & 1, sub & 1, p ^ 1, 1, launches, st));
        CK(launch_substep(A, last, last, p ^ 1, 0, launches, st));
    }
    if (ev) CK(cudaEventRecord(ev[2], st));
    if (overlap) {
        // lists of the next step (parity p ^ 1 reads buffer p): the histories are final
        // after this step's last contact sums, the positions after its last predictor
        CK(cudaEventRecord(s->fork_ev, st));
        CK(cudaStreamWaitEvent(s->side, s->fork_ev, 0));
        CK(launch_rebuild(A, p ^ 1, p, last, s->scan_partial, s->side, launches));
        CK(cudaEventRecord(s->join_ev, s->side));
    }
    if (s->lattice) {
        LbmArgs la = lbm_args(s, p, p ^ 1, last);
        CK(cudaMemsetAsync(s->tile_count, 0, sizeof(int) * (size_t)s->ntiles, st));
        if (n > 0) {
            CK(cudaMemsetAsync(s->P.Fh, 0, sizeof(double) * 6 * (size_t)s->P.cap, st));
            CK(launch_bin(la, n, s->tile_count, s->tile_ids, st));
            *launches += 1;
        }
        if (ev) CK(cudaEventRecord(ev[3], st));
        CK(launch_psm(la, s->staged ? &s->maps[p] : nullptr, s->p.storage, st));
        *launches += 1;
    } else if (ev) {
        CK(cudaEventRecord(ev[3], st));
    }
    if (ev) CK(cudaEventRecord(ev[4], st));
    if (overlap) CK(cudaStreamWaitEvent(st, s->join_ev, 0));
    if (n > 0) {
        CK(launch_final(A, last, s->lattice ? 1 : 0, st));
        *launches += 1;
    }
    if (ev) CK(cudaEventRecord(ev[5], st));
    return cudaSuccess;
}

static cudaError_t capture(ledds_sim_s* s, int p, int nsteps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    int launches = 0;
    CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < nsteps && e == cudaSuccess; ++q) e = enqueue_step(s, p ^ (q & 1), s->cap_stream, &launches, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    if (e2 != cudaSuccess) return e2;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    s->launches_per_step = launches / nsteps;
    return e;
}

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" {

int ledds_version(void) { return 1; }

const char* ledds_strerror(int code) {
    switch (code) {
        case LEDDS_OK: return "ok";
        case LEDDS_ERR_INVALID_ARG: return "invalid argument";
        case LEDDS_ERR_CAPACITY: return "capacity exceeded";
        case LEDDS_ERR_NAN: return "non-finite values detected";
        case LEDDS_ERR_TIMEOUT: return "device wait timed out";
        case LEDDS_ERR_CUDA: return "CUDA runtime error";
        case LEDDS_ERR_STATE: return "invalid state for this call";
        default: return "unknown error";
    }
}

int ledds_params_default(ledds_params* p) {
    if (!p) return LEDDS_ERR_INVALID_ARG;
    memset(p, 0, sizeof(*p));
    p->tau = 0.8;
    p->storage = LEDDS_STORE_F32;
    p->storage_scale_log2 = 10;
    p->voxel = LEDDS_VOXEL_DISTANCE;
    p->subdiv_n = 10;
    p->law = LEDDS_LAW_LINEAR;
    p->n_sub = 1;
    p->rho_f = 1.0;
    p->k_n = 1000.0;
    p->k_t = 1000.0 * 2.0 / 7.0;
    p->young = 1.0e4;
    p->poisson = 0.3;
    p->restitution = 0.7;
    p->friction = 0.4;
    p->skin = 0.5;
    p->dem_h = 0.0;
    p->ell_max_iter = 60;
    p->ell_tol = 1e-6;
    p->force_fp32 = 1;
    p->collision = LEDDS_COLLIDE_BGK;
    p->orient = LEDDS_ORIENT_TRIAD;
    p->pattern = LEDDS_PATTERN_AB;
    p->index64 = 0;
    p->psm_route = 0;
    p->ell_screen = 1;
    return LEDDS_OK;
}

int ledds_workspace_size(const ledds_dims* d, const ledds_params* p, size_t* bytes) {
    int rc = check_args(d, p);
    if (rc != LEDDS_OK) return rc;
    if (!bytes) return LEDDS_ERR_INVALID_ARG;
    *bytes = layout(nullptr, d, p, nullptr);
    return LEDDS_OK;
}

int ledds_create(const ledds_dims* d, const ledds_params* p, void* d_workspace, size_t bytes,
                 void* stream, ledds_sim_t* out) {
    int rc = check_args(d, p);
    if (rc != LEDDS_OK) return rc;
    if (!out || !d_workspace || ((uintptr_t)d_workspace & 255)) return LEDDS_ERR_INVALID_ARG;
    size_t need = layout(nullptr, d, p, nullptr);
    if (bytes < need) return LEDDS_ERR_INVALID_ARG;
    ledds_sim_s* s = new ledds_sim_s();
    s->d = *d;
    s->p = *p;
    s->stream = (cudaStream_t)stream;
    s->ws = (char*)d_workspace;
    s->ws_bytes = bytes;
    memset(s->uw, 0, sizeof(s->uw));
    domain(d, s->lo, s->hi, s->L);
    layout(s, d, p, s->ws);
    {
        int dev = 0, n_sm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n_sm > 0)
            s->sms = n_sm;
    }
    if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->join_ev, cudaEventDisableTiming) != cudaSuccess) {
        if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
        if (s->side) cudaStreamDestroy(s->side);
        if (s->fork_ev) cudaEventDestroy(s->fork_ev);
        if (s->join_ev) cudaEventDestroy(s->join_ev);
        delete s;
        return LEDDS_ERR_CUDA;
    }
    cudaError_t e = cudaMemsetAsync(s->ws, 0, need - 256, s->stream);
    if (e == cudaSuccess && s->lattice) {
        LbmArgs a = lbm_args(s, 0, 0, 0);
        e = launch_init(a, s->p.storage, nullptr, nullptr, nullptr, s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s->cap_stream);
        cudaStreamDestroy(s->side);
        cudaEventDestroy(s->fork_ev);
        cudaEventDestroy(s->join_ev);
        delete s;
        return LEDDS_ERR_CUDA;
    }
    *out = s;
    return LEDDS_OK;
}

int ledds_destroy(ledds_sim_t s) {
    if (!s) return LEDDS_ERR_INVALID_ARG;
    if (s->in_batch) return LEDDS_ERR_STATE;  // owned by its batch
    drop_graphs(s);
    if (s->ev_made)
        for (int q = 0; q <= NSTAGE; ++q) cudaEventDestroy(s->ev[q]);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->fork_ev) cudaEventDestroy(s->fork_ev);
    if (s->join_ev) cudaEventDestroy(s->join_ev);
    delete s;
    return LEDDS_OK;
}

int ledds_set_wall_velocity(ledds_sim_t s, int axis, int side, const double u[3]) {
    if (!s || !u || axis < 0 || axis > 2 || side < 0 || side > 1) return LEDDS_ERR_INVALID_ARG;
    if (s->d.periodic[axis]) return LEDDS_ERR_INVALID_ARG;
    float old[3][2][3];
    for (int q = 0; q < 3; ++q)
        for (int e = 0; e < 2; ++e)
            for (int c = 0; c < 3; ++c) old[q][e][c] = (float)s->uw[q][e][c];
    for (int c = 0; c < 3; ++c) s->uw[axis][side][c] = u[c];
    drop_graphs(s);
    if (s->lattice) {
        // the current pre-collision populations stay as they are
        LbmArgs a = lbm_args(s, s->parity, s->parity, 0);
        if (a.aa != PSM_AA_EVEN && launch_rebase(a, s->p.storage, old, s->stream) != cudaSuccess)
            return LEDDS_ERR_CUDA;
    }
    return LEDDS_OK;
}

int ledds_set_forcing(ledds_sim_t s, const double gravity[3], const double fluid_force[3]) {
    if (!s) return LEDDS_ERR_INVALID_ARG;
    if (gravity)
        for (int c = 0; c < 3; ++c) s->p.gravity[c] = gravity[c];
    if (fluid_force)
        for (int c = 0; c < 3; ++c) s->p.fluid_force[c] = fluid_force[c];
    drop_graphs(s);
    return LEDDS_OK;
}

int ledds_init_fluid(ledds_sim_t s, const float* d_rho, const float* d_u) {
    if (!s) return LEDDS_ERR_INVALID_ARG;
    if (!s->lattice) return LEDDS_ERR_STATE;
    LbmArgs a = lbm_args(s, s->parity, s->parity, 0);
    return launch_init(a, s->p.storage, d_rho, d_u, nullptr, s->stream) == cudaSuccess ? LEDDS_OK
                                                                                       : LEDDS_ERR_CUDA;
}

int ledds_init_populations(ledds_sim_t s, const float* d_f) {
    if (!s || !d_f) return LEDDS_ERR_INVALID_ARG;
    if (!s->lattice) return LEDDS_ERR_STATE;
    LbmArgs a = lbm_args(s, s->parity, s->parity, 0);
    return launch_init(a, s->p.storage, nullptr, nullptr, d_f, s->stream) == cudaSuccess ? LEDDS_OK
                                                                                       : LEDDS_ERR_CUDA;
}

static int upload_rows(ledds_sim_t s, double* dst, const double* src, int rows, int n, int on_device) {
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpy2DAsync(dst, sizeof(double) * s->P.cap, src, sizeof(double) * n,
                                      sizeof(double) * n, rows, kind, s->stream);
    return e == cudaSuccess ? LEDDS_OK : LEDDS_ERR_CUDA;
}

int ledds_set_particles(ledds_sim_t s, int n, const ledds_particle* h) {
    if (!s || n < 0 || n > s->d.max_particles || (n > 0 && !h)) return LEDDS_ERR_INVALID_ARG;
    std::vector<double> st(18 * (size_t)(n > 0 ? n : 1)), radius(n + 1), semi(3 * (size_t)n + 3), bound(n + 1),
        mass(n + 1), inertia(3 * (size_t)n + 3), gfac(n + 1), acc(3 * (size_t)n + 3);
    std::vector<int> shape(n + 1);
    double bmax = 0.0;
    for (int k = 0; k < n; ++k) {
        const ledds_particle& q = h[k];
        if (q.shape != LEDDS_SPHERE && q.shape != LEDDS_ELLIPSOID) return LEDDS_ERR_INVALID_ARG;
        if (!(q.density > 0.0)) return LEDDS_ERR_INVALID_ARG;
        double V, m, I[3], b;
        if (q.shape == LEDDS_SPHERE) {
            double R = q.radius;
            if (!(R > 0.0)) return LEDDS_ERR_INVALID_ARG;
            V = 4.0 / 3.0 * kPi * R * R * R;
            m = q.density * V;
            for (int a = 0; a < 3; ++a) I[a] = 2.0 * m * R * R / 5.0;
            radius[k] = R;
            b = R;
            for (int a = 0; a < 3; ++a) semi[a * (size_t)n + k] = R;
        } else {
            double A = q.semi[0], B = q.semi[1], C = q.semi[2];
            if (!(A > 0.0 && B > 0.0 && C > 0.0)) return LEDDS_ERR_INVALID_ARG;
            V = 4.0 / 3.0 * kPi * A * B * C;
            m = q.density * V;
            I[0] = m * (B * B + C * C) / 5.0;
            I[1] = m * (A * A + C * C) / 5.0;
            I[2] = m * (A * A + B * B) / 5.0;
            b = fmax(A, fmax(B, C));
            radius[k] = b;
            for (int a = 0; a < 3; ++a) semi[a * (size_t)n + k] = q.semi[a];
        }
        // orthonormal triad
        const double* t = q.triad;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double dd = t[3 * i] * t[3 * j] + t[3 * i + 1] * t[3 * j + 1] + t[3 * i + 2] * t[3 * j + 2];
                if (fabs(dd - (i == j ? 1.0 : 0.0)) > 1e-6) return LEDDS_ERR_INVALID_ARG;
            }
        bound[k] = b;
        bmax = fmax(bmax, b);
        mass[k] = m;
        for (int a = 0; a < 3; ++a) inertia[a * (size_t)n + k] = I[a];
        gfac[k] = 1.0 - s->p.rho_f / q.density;
        shape[k] = q.shape;
        for (int a = 0; a < 3; ++a) {
            st[(SP + a) * (size_t)n + k] = q.pos[a];
            st[(SV + a) * (size_t)n + k] = q.vel[a];
            st[(SW + a) * (size_t)n + k] = q.omg[a];
            acc[a * (size_t)n + k] = s->p.gravity[a] * gfac[k];
        }
        for (int m9 = 0; m9 < 9; ++m9) st[(ST + m9) * (size_t)n + k] = t[m9];
    }
    // The candidate search covers the 27 neighbouring cells, so a cell must be at least
    // as wide as the largest interaction range; periodic boxes must exceed twice it.
    double range = 2.0 * bmax + s->p.skin;
    for (int a = 0; a < 3; ++a) {
        if (n > 0 && s->gh[a] < range) return LEDDS_ERR_INVALID_ARG;
        if (n > 0 && s->d.periodic[a] && s->L[a] <= 2.0 * range) return LEDDS_ERR_INVALID_ARG;
    }
    if (s->lattice && n > 0) {
        int n3[3] = {s->d.nx, s->d.ny, s->d.nz};
        double reach = bmax + 1.0 + (cbrt(3.0 / (4.0 * kPi)));
        for (int a = 0; a < 3; ++a)
            if (s->d.periodic[a] && 2.0 * reach + 2.0 >= n3[a]) return LEDDS_ERR_INVALID_ARG;
    }
    s->P.n = n;
    s->max_bound = bmax;
    s->lists_ready = false;
    s->any_ellipsoid = 0;
    for (int k = 0; k < n; ++k) s->any_ellipsoid |= shape[k] == LEDDS_ELLIPSOID;
    drop_graphs(s);
    if (n > 0) {
        int rc;
        if ((rc = upload_rows(s, s->P.st[0], st.data(), 18, n, 0)) != LEDDS_OK) return rc;
        if ((rc = upload_rows(s, s->P.st[1], st.data(), 18, n, 0)) != LEDDS_OK) return rc;
        if ((rc = upload_rows(s, s->P.radius, radius.data(), 1, n, 0)) != LEDDS_OK) return rc;
        if ((rc = upload_rows(s, s->P.semi, semi.data(), 3, n, 0)) != LEDDS_OK) return rc;
        if ((rc = upload_rows(s, s->P.bound, bound.data(), 1, n, 0)) != LEDDS_OK) return rc;
        if ((rc = upload_rows(s, s->P.mass, mass.data(), 1, n, 0)) != LEDDS_OK) return rc;
        if ((rc = upload_rows(s, s->P.inertia, inertia.data(), 3, n, 0)) != LEDDS_OK) return rc;
        if ((rc = upload_rows(s, s->P.gfac, gfac.data(), 1, n, 0)) != LEDDS_OK) return rc;
        if ((rc = upload_rows(s, s->P.acc, acc.data(), 3, n, 0)) != LEDDS_OK) return rc;
        if (cudaMemcpyAsync(s->P.shape, shape.data(), sizeof(int) * n, cudaMemcpyHostToDevice,
                            s->stream) != cudaSuccess)
            return LEDDS_ERR_CUDA;
    }
    size_t c3 = sizeof(double) * 3 * (size_t)s->P.cap;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemsetAsync(s->P.alpha, 0, c3, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->P.Fc, 0, c3, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->P.Mc, 0, c3, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->P.Fh, 0, 2 * c3, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->P.Fhp, 0, 2 * c3, s->stream);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMemsetAsync(s->ncand[b], 0, sizeof(int) * s->P.cap, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->whist, 0, sizeof(double) * 18 * (size_t)s->P.cap, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LEDDS_OK : LEDDS_ERR_CUDA;
}

int ledds_write_kinematics(ledds_sim_t s, const double* state, int on_device) {
    if (!s || !state) return LEDDS_ERR_INVALID_ARG;
    if (s->P.n == 0) return LEDDS_OK;
    int rc = upload_rows(s, s->P.st[0], state, 18, s->P.n, on_device);
    s->lists_ready = false;  // new positions: the next step builds its lists first
    if (rc == LEDDS_OK && !on_device && cudaStreamSynchronize(s->stream) != cudaSuccess) return LEDDS_ERR_CUDA;
    return rc;
}

int ledds_step(ledds_sim_t s, int n_steps) {
    if (!s || n_steps < 0) return LEDDS_ERR_INVALID_ARG;
    if (s->in_batch) return LEDDS_ERR_STATE;  // members advance with ledds_batch_step
    if (s->profiling) {
        if (!s->ev_made) {
            for (int q = 0; q <= NSTAGE; ++q)
                if (cudaEventCreate(&s->ev[q]) != cudaSuccess) return LEDDS_ERR_CUDA;
            s->ev_made = true;
        }
        for (int k = 0; k < n_steps; ++k) {
            int launches = 0;
            if (enqueue_step(s, s->parity, s->stream, &launches, s->ev) != cudaSuccess) return LEDDS_ERR_CUDA;
            if (cudaEventSynchronize(s->ev[NSTAGE]) != cudaSuccess) return LEDDS_ERR_CUDA;
            for (int q = 0; q < NSTAGE; ++q) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, s->ev[q], s->ev[q + 1]);
                s->prof_ms[q] += ms;
            }
            s->prof_steps++;
            s->prof_launches += launches;
            s->launches_per_step = launches;
            s->parity ^= 1;
            s->steps++;
        }
        s->lists_ready = false;  // profiled steps rebuild at their start, not for the next one
        return LEDDS_OK;
    }
    if (n_steps > 0 && s->lattice && s->P.n > 0 && !s->lists_ready) {
        // the first step after new positions: its lists, as a step of the serial order
        // builds them (one captured graph per parity: host-driven loops that rewrite the
        // kinematics every step take this path every step)
        const int p = s->parity;
        if (!s->grb[p]) {
            DemArgs A = dem_args(s);
            int launches = 0;
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return LEDDS_ERR_CUDA;
            cudaError_t e = launch_rebuild(A, p, p ^ 1, 0, s->scan_partial, s->cap_stream, &launches);
            cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &g);
            if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&s->grb[p], g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess || e2 != cudaSuccess) return LEDDS_ERR_CUDA;
        }
        if (cudaGraphLaunch(s->grb[p], s->stream) != cudaSuccess) return LEDDS_ERR_CUDA;
    }
    s->lists_ready = true;  // every graph step ends with the rebuild for the next
    int left = n_steps;
    while (left > 0) {
        int p = s->parity;
        if (left >= 2) {
            if (!s->g2[p] && capture(s, p, 2, &s->g2[p]) != cudaSuccess) return LEDDS_ERR_CUDA;
            if (cudaGraphLaunch(s->g2[p], s->stream) != cudaSuccess) return LEDDS_ERR_CUDA;
            left -= 2;
            s->steps += 2;
        } else {
            if (!s->g1[p] && capture(s, p, 1, &s->g1[p]) != cudaSuccess) return LEDDS_ERR_CUDA;
            if (cudaGraphLaunch(s->g1[p], s->stream) != cudaSuccess) return LEDDS_ERR_CUDA;
            left -= 1;
            s->steps += 1;
            s->parity ^= 1;
        }
    }
    return LEDDS_OK;
}

int ledds_sync(ledds_sim_t s) {
    if (!s) return LEDDS_ERR_INVALID_ARG;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? LEDDS_OK : LEDDS_ERR_CUDA;
}

int ledds_get_status(ledds_sim_t s, ledds_status* st) {
    if (!s || !st) return LEDDS_ERR_INVALID_ARG;
    DevStatus h;
    if (cudaMemcpyAsync(&h, s->status, sizeof(h), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return LEDDS_ERR_CUDA;
    st->steps = s->steps;
    st->tile_overflow = h.tile_overflow;
    st->cand_overflow = h.cand_overflow;
    st->solids_overflow = h.solids_overflow;
    st->skin_violation = h.skin_violation;
    st->ell_nonconverged = h.ell_nonconverged;
    st->nan_detected = h.nan_detected;
    st->n_particles = s->P.n;
    st->launches_per_step = s->launches_per_step;
    st->wait_timeout = h.wait_timeout;
    st->psm_staged = s->staged ? 1 : 0;
    if (h.nan_detected) return LEDDS_ERR_NAN;
    if (h.wait_timeout) return LEDDS_ERR_TIMEOUT;
    if (h.tile_overflow || h.cand_overflow) return LEDDS_ERR_CAPACITY;
    return LEDDS_OK;
}

int ledds_read_fields(ledds_sim_t s, float* d_rho, float* d_u) {
    if (!s) return LEDDS_ERR_INVALID_ARG;
    if (!s->lattice) return LEDDS_ERR_STATE;
    LbmArgs a = lbm_args(s, s->parity, s->parity, 0);
    return launch_read(a, s->p.storage, d_rho, d_u, nullptr, 0, s->stream) == cudaSuccess ? LEDDS_OK
                                                                                       : LEDDS_ERR_CUDA;
}

int ledds_read_populations(ledds_sim_t s, float* d_f, int which) {
    if (!s || !d_f || which < 0 || which > 1) return LEDDS_ERR_INVALID_ARG;
    if (!s->lattice) return LEDDS_ERR_STATE;
    LbmArgs a = lbm_args(s, s->parity, s->parity, 0);
    return launch_read(a, s->p.storage, nullptr, nullptr, d_f, which, s->stream) == cudaSuccess
               ? LEDDS_OK
               : LEDDS_ERR_CUDA;
}

int ledds_read_particles(ledds_sim_t s, double* state, int on_device) {
    if (!s || !state) return LEDDS_ERR_INVALID_ARG;
    int n = s->P.n;
    if (n == 0) return LEDDS_OK;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpy2DAsync(state, sizeof(double) * n, s->P.st[0], sizeof(double) * s->P.cap,
                                      sizeof(double) * n, 18, kind, s->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LEDDS_OK : LEDDS_ERR_CUDA;
}

int ledds_read_forces(ledds_sim_t s, double* d_Fh, double* d_Mh, double* d_Fc, double* d_Mc) {
    if (!s) return LEDDS_ERR_INVALID_ARG;
    int n = s->P.n;
    if (n == 0) return LEDDS_OK;
    double* src[4] = {s->P.Fh, s->P.Mh, s->P.Fc, s->P.Mc};
    double* dst[4] = {d_Fh, d_Mh, d_Fc, d_Mc};
    for (int q = 0; q < 4; ++q) {
        if (!dst[q]) continue;
        if (cudaMemcpy2DAsync(dst[q], sizeof(double) * n, src[q], sizeof(double) * s->P.cap,
                              sizeof(double) * n, 3, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
            return LEDDS_ERR_CUDA;
    }
    return LEDDS_OK;
}

int ledds_read_pairs(ledds_sim_t s, uint64_t* d_keys, int cap, int* n_out) {
    if (!s || !n_out || cap < 0 || (cap > 0 && !d_keys)) return LEDDS_ERR_INVALID_ARG;
    *n_out = 0;
    if (s->P.n == 0) return LEDDS_OK;
    DemArgs A = dem_args(s);
    if (launch_pairs(A, s->parity, s->pair_cnt, s->pair_off, s->scan_partial,
                     (unsigned long long*)d_keys, cap, s->stream) != cudaSuccess)
        return LEDDS_ERR_CUDA;
    uint32_t tot = 0;
    if (cudaMemcpyAsync(&tot, s->pair_off + s->P.n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return LEDDS_ERR_CUDA;
    *n_out = (int)tot;
    return LEDDS_OK;
}

int ledds_read_cell_keys(ledds_sim_t s, uint32_t* d_keys, int32_t* d_sorted_ids, int grid_n[3]) {
    if (!s) return LEDDS_ERR_INVALID_ARG;
    if (s->in_batch) return LEDDS_ERR_STATE;  // a batch searches candidates directly, without a cell list
    int n = s->P.n;
    if (grid_n)
        for (int a = 0; a < 3; ++a) grid_n[a] = s->gn[a];
    if (n == 0) return LEDDS_OK;
    if (d_keys && cudaMemcpyAsync(d_keys, s->keys, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
        return LEDDS_ERR_CUDA;
    if (d_sorted_ids &&
        cudaMemcpyAsync(d_sorted_ids, s->sorted, sizeof(int) * n, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
        return LEDDS_ERR_CUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? LEDDS_OK : LEDDS_ERR_CUDA;
}

int ledds_voxelize(ledds_sim_t s, float* d_beta, int32_t* d_ids, int32_t* d_nsolid) {
    if (!s || !d_beta || !d_ids || !d_nsolid) return LEDDS_ERR_INVALID_ARG;
    if (!s->lattice) return LEDDS_ERR_STATE;
    LbmArgs a = lbm_args(s, s->parity, s->parity, 0);
    if (cudaMemsetAsync(s->tile_count, 0, sizeof(int) * (size_t)s->ntiles, s->stream) != cudaSuccess)
        return LEDDS_ERR_CUDA;
    if (launch_bin(a, s->P.n, s->tile_count, s->tile_ids, s->stream) != cudaSuccess) return LEDDS_ERR_CUDA;
    if (launch_voxelize(a, d_beta, d_ids, d_nsolid, s->stream) != cudaSuccess) return LEDDS_ERR_CUDA;
    return LEDDS_OK;
}

int ledds_set_profiling(ledds_sim_t s, int on) {
    if (!s) return LEDDS_ERR_INVALID_ARG;
    s->profiling = on != 0;
    return LEDDS_OK;
}

int ledds_read_profile(ledds_sim_t s, double ms[5], long long* steps, long long* launches) {
    if (!s) return LEDDS_ERR_INVALID_ARG;
    if (ms)
        for (int q = 0; q < NSTAGE; ++q) ms[q] = s->prof_ms[q];
    if (steps) *steps = s->prof_steps;
    if (launches) *launches = s->prof_launches;
    for (int q = 0; q < NSTAGE; ++q) s->prof_ms[q] = 0.0;
    s->prof_steps = s->prof_launches = 0;
    return LEDDS_OK;
}

// Checkpoint: a small header with the host-side state, then the whole workspace image.
struct CkptHeader {
    char magic[8];
    int version;
    ledds_dims d;
    ledds_params p;
    int n, parity;
    long long steps;
    double uw[3][2][3];
    size_t ws_used;
    double max_bound;  // derived from the particles at upload; not recomputed on load
    int any_ellipsoid;
};

int ledds_save(ledds_sim_t s, void* h_buf, size_t* bytes) {
    if (!s || !bytes) return LEDDS_ERR_INVALID_ARG;
    size_t used = layout(nullptr, &s->d, &s->p, nullptr) - 256;
    size_t need = sizeof(CkptHeader) + used;
    if (!h_buf) {
        *bytes = need;
        return LEDDS_OK;
    }
    if (*bytes < need) return LEDDS_ERR_INVALID_ARG;
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "LEDDSCK2", 8);
    hd.version = 2;
    hd.d = s->d;
    hd.p = s->p;
    hd.n = s->P.n;
    hd.parity = s->parity;
    hd.steps = s->steps;
    memcpy(hd.uw, s->uw, sizeof(hd.uw));
    hd.ws_used = used;
    hd.max_bound = s->max_bound;
    hd.any_ellipsoid = s->any_ellipsoid;
    memcpy(h_buf, &hd, sizeof(hd));
    if (cudaMemcpyAsync((char*)h_buf + sizeof(hd), s->ws, used, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return LEDDS_ERR_CUDA;
    *bytes = need;
    return LEDDS_OK;
}

// Effective candidate and tile capacities of a dims record (0 selects the defaults).
static int cand_cap_of(const ledds_dims& d) { return d.cand_cap > 0 ? d.cand_cap : 32; }
static int tile_cap_of(const ledds_dims& d) { return d.tile_cap > 0 ? d.tile_cap : 64; }

// A checkpoint taken with smaller candidate or tile capacities, copied into this
// simulation's layout: arrays that do not depend on the capacities whole, the candidate
// lists and their tangential histories row by row (one row per particle, the new rows
// longer), and nothing of the lists every step rebuilds (tile lists, pair-once lists).
static cudaError_t load_resized(ledds_sim_t s, const CkptHeader& hd, const char* img) {
    ledds_sim_s o;  // the checkpoint's layout, as offsets from a stand-in base
    char* const base = reinterpret_cast<char*>(4096);
    layout(&o, &hd.d, &hd.p, base);
    cudaError_t e = cudaSuccess;
    auto whole = [&](void* dst, const void* old, size_t bytes) {
        if (e == cudaSuccess && bytes)
            e = cudaMemcpyAsync(dst, img + ((const char*)old - base), bytes, cudaMemcpyHostToDevice, s->stream);
    };
    auto rows = [&](void* dst, const void* old, size_t row_old, size_t row_new, size_t nrows) {
        if (e == cudaSuccess && nrows)
            e = cudaMemcpy2DAsync(dst, row_new, img + ((const char*)old - base), row_old, row_old, nrows,
                                  cudaMemcpyHostToDevice, s->stream);
    };
    const size_t N19 = (size_t)s->N * 19 * storage_bytes(s->p.storage);
    whole(s->pop[0], o.pop[0], N19);
    if (s->pop[1] != s->pop[0]) whole(s->pop[1], o.pop[1], N19);
    const size_t c = (size_t)s->P.cap, d8 = sizeof(double);
    for (int b = 0; b < 2; ++b) whole(s->P.st[b], o.P.st[b], 18 * c * d8);
    whole(s->P.acc, o.P.acc, 3 * c * d8);
    whole(s->P.alpha, o.P.alpha, 3 * c * d8);
    whole(s->P.Fc, o.P.Fc, 3 * c * d8);
    whole(s->P.Mc, o.P.Mc, 3 * c * d8);
    whole(s->P.Fh, o.P.Fh, 6 * c * d8);    // Fh and Mh
    whole(s->P.Fhp, o.P.Fhp, 6 * c * d8);  // Fhp and Mhp
    whole(s->P.pos_build, o.P.pos_build, 3 * c * d8);
    whole(s->P.radius, o.P.radius, c * d8);
    whole(s->P.semi, o.P.semi, 3 * c * d8);
    whole(s->P.bound, o.P.bound, c * d8);
    whole(s->P.mass, o.P.mass, c * d8);
    whole(s->P.inertia, o.P.inertia, 3 * c * d8);
    whole(s->P.gfac, o.P.gfac, c * d8);
    whole(s->P.shape, o.P.shape, c * sizeof(int));
    whole(s->keys, o.keys, c * sizeof(uint32_t));
    whole(s->rank, o.rank, c * sizeof(int));
    whole(s->sorted, o.sorted, c * sizeof(int));
    whole(s->cell_count, o.cell_count, ((size_t)s->G + 1) * sizeof(uint32_t));
    whole(s->cell_start, o.cell_start, ((size_t)s->G + 1) * sizeof(uint32_t));
    const size_t oc = (size_t)o.ccap, nc = (size_t)s->ccap;
    for (int b = 0; b < 2; ++b) {
        rows(s->cand[b], o.cand[b], oc * sizeof(int), nc * sizeof(int), c);
        whole(s->ncand[b], o.ncand[b], c * sizeof(int));
        rows(s->hist[b], o.hist[b], oc * 3 * d8, nc * 3 * d8, c);
    }
    whole(s->whist, o.whist, 18 * c * d8);
    whole(s->status, o.status, sizeof(DevStatus));
    return e;
}

int ledds_load(ledds_sim_t s, const void* h_buf, size_t bytes) {
    if (!s || !h_buf || bytes < sizeof(CkptHeader)) return LEDDS_ERR_INVALID_ARG;
    CkptHeader hd;
    memcpy(&hd, h_buf, sizeof(hd));
    size_t used = layout(nullptr, &s->d, &s->p, nullptr) - 256;
    if (memcmp(hd.magic, "LEDDSCK2", 8) != 0 || hd.p.storage != s->p.storage || hd.p.pattern != s->p.pattern)
        return LEDDS_ERR_INVALID_ARG;
    // the same dims, or the same but for larger candidate or tile capacities here
    ledds_dims same = hd.d;
    same.cand_cap = s->d.cand_cap;
    same.tile_cap = s->d.tile_cap;
    if (memcmp(&same, &s->d, sizeof(ledds_dims)) != 0) return LEDDS_ERR_INVALID_ARG;
    const bool resized = memcmp(&hd.d, &s->d, sizeof(ledds_dims)) != 0;
    if (resized && (cand_cap_of(hd.d) > cand_cap_of(s->d) || tile_cap_of(hd.d) > tile_cap_of(s->d)))
        return LEDDS_ERR_INVALID_ARG;
    const size_t used_old = resized ? layout(nullptr, &hd.d, &hd.p, nullptr) - 256 : used;
    if (hd.ws_used != used_old || bytes < sizeof(hd) + used_old) return LEDDS_ERR_INVALID_ARG;
    const char* img = (const char*)h_buf + sizeof(hd);
    cudaError_t e = resized ? load_resized(s, hd, img)
                            : cudaMemcpyAsync(s->ws, img, used, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess || cudaStreamSynchronize(s->stream) != cudaSuccess) return LEDDS_ERR_CUDA;
    s->p = hd.p;
    s->P.n = hd.n;
    // (tile lists are rebuilt by every step; the leading rebuild of the next step
    // rebuilds the candidate lists from the loaded positions and histories)
    s->parity = hd.parity;
    s->steps = hd.steps;
    memcpy(s->uw, hd.uw, sizeof(hd.uw));
    s->max_bound = hd.max_bound;
    s->any_ellipsoid = hd.any_ellipsoid;
    s->lists_ready = false;
    drop_graphs(s);
    return LEDDS_OK;
}

// ------------------------------------------------------------------------------------
// Batches: many independent simulations advanced by one set of launches per step.
// ------------------------------------------------------------------------------------
struct ledds_batch_s {
    int nsim = 0;
    std::vector<ledds_sim_s*> sims;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    int storage = 0, parity = 0, nblocks = 0;
    long long steps = 0;
    LbmArgs* d_largs[2] = {nullptr, nullptr};
    DemArgs* d_dargs = nullptr;
    int *d_tile_start = nullptr, *d_np = nullptr, *d_poff = nullptr, *d_counter = nullptr;
    int nchunks = 0;
    std::vector<BatchChunk> chunks[2];  // PSM launch arguments per batch parity
    int ctas_per_sm = 0, sms = 1;        // persistent PSM grid = ctas_per_sm x SMs
    int order = 0;                       // PSM work order: 0 member order, 1 largest first
    int tz = TILE_Z;                     // tile depth of every member
    bool sphd = false;                   // every member: distance-fraction spheres, no wrap
    cudaGraphExec_t g1[2] = {nullptr, nullptr}, g2[2] = {nullptr, nullptr};
    std::vector<long long> versions;
};

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static int batch_layout(int nsim, const ledds_dims* dims, const ledds_params* params, std::vector<size_t>* offs,
                        size_t* total) {
    if (nsim <= 0 || !dims || !params) return LEDDS_ERR_INVALID_ARG;
    size_t off = 0;
    for (int i = 0; i < nsim; ++i) {
        int rc = check_args(&dims[i], &params[i]);
        if (rc != LEDDS_OK) return rc;
        if (dims[i].nx <= 0) return LEDDS_ERR_INVALID_ARG;  // every member has a lattice
        if (params[i].storage != params[0].storage) return LEDDS_ERR_INVALID_ARG;
        if (params[i].collision != params[0].collision) return LEDDS_ERR_INVALID_ARG;
        if (params[i].pattern != LEDDS_PATTERN_AB) return LEDDS_ERR_INVALID_ARG;  // batches use two lattices
        if (params[i].index64 || 19.0 * dims[i].nx * dims[i].ny * dims[i].nz >= 2147483647.0)
            return LEDDS_ERR_INVALID_ARG;  // and 32-bit population offsets
        if (dims[i].max_particles > 4096) return LEDDS_ERR_INVALID_ARG;  // direct candidate search
        if (offs) offs->push_back(off);
        off = align256(off + layout(nullptr, &dims[i], &params[i], nullptr));
    }
    off = align256(off + 2 * sizeof(LbmArgs) * nsim);
    off = align256(off + sizeof(DemArgs) * nsim);
    const int nchunks = (nsim + BATCH_CHUNK - 1) / BATCH_CHUNK;
    off = align256(off + sizeof(int) * (3 * nsim + 1 + nchunks));
    *total = off + 256;
    return LEDDS_OK;
}

int ledds_batch_workspace_size(int nsim, const ledds_dims* dims, const ledds_params* params, size_t* bytes) {
    if (!bytes) return LEDDS_ERR_INVALID_ARG;
    return batch_layout(nsim, dims, params, nullptr, bytes);
}

static void batch_drop_graphs(ledds_batch_s* b) {
    for (int q = 0; q < 2; ++q) {
        if (b->g1[q]) cudaGraphExecDestroy(b->g1[q]);
        if (b->g2[q]) cudaGraphExecDestroy(b->g2[q]);
        b->g1[q] = b->g2[q] = nullptr;
    }
}

int ledds_batch_destroy(ledds_batch_t b) {
    if (!b) return LEDDS_ERR_INVALID_ARG;
    batch_drop_graphs(b);
    for (auto* s : b->sims) {
        s->in_batch = false;
        ledds_destroy(s);
    }
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return LEDDS_OK;
}

int ledds_batch_create(int nsim, const ledds_dims* dims, const ledds_params* params, void* d_workspace,
                       size_t bytes, void* stream, ledds_batch_t* out) {
    std::vector<size_t> offs;
    size_t need = 0;
    int rc = batch_layout(nsim, dims, params, &offs, &need);
    if (rc != LEDDS_OK) return rc;
    if (!out || !d_workspace || ((uintptr_t)d_workspace & 255) || bytes < need) return LEDDS_ERR_INVALID_ARG;
    ledds_batch_s* b = new ledds_batch_s();
    b->nsim = nsim;
    b->stream = (cudaStream_t)stream;
    b->storage = params[0].storage;
    char* ws = (char*)d_workspace;
    for (int i = 0; i < nsim; ++i) {
        ledds_sim_t s = nullptr;
        size_t sz = layout(nullptr, &dims[i], &params[i], nullptr);
        rc = ledds_create(&dims[i], &params[i], ws + offs[i], sz, stream, &s);
        if (rc != LEDDS_OK) {
            ledds_batch_destroy(b);
            return rc;
        }
        s->in_batch = true;
        b->sims.push_back(s);
    }
    size_t off = align256(offs.back() + layout(nullptr, &dims[nsim - 1], &params[nsim - 1], nullptr));
    b->d_largs[0] = reinterpret_cast<LbmArgs*>(ws + off);
    b->d_largs[1] = b->d_largs[0] + nsim;
    off = align256(off + 2 * sizeof(LbmArgs) * nsim);
    b->d_dargs = reinterpret_cast<DemArgs*>(ws + off);
    off = align256(off + sizeof(DemArgs) * nsim);
    b->d_tile_start = reinterpret_cast<int*>(ws + off);
    b->d_np = b->d_tile_start + nsim + 1;
    b->d_poff = b->d_np + nsim;
    b->d_counter = b->d_poff + nsim;
    b->nchunks = (nsim + BATCH_CHUNK - 1) / BATCH_CHUNK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->sms = sms > 0 ? sms : 1;
    b->ctas_per_sm = psm_batch_ctas_per_sm();
    b->nblocks = b->ctas_per_sm * b->sms;  // one wave of resident CTAs
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        ledds_batch_destroy(b);
        return LEDDS_ERR_CUDA;
    }
    *out = b;
    return LEDDS_OK;
}

int ledds_batch_sim(ledds_batch_t b, int i, ledds_sim_t* out) {
    if (!b || !out || i < 0 || i >= b->nsim) return LEDDS_ERR_INVALID_ARG;
    *out = b->sims[i];
    return LEDDS_OK;
}

// Upload the per-member kernel arguments (both batch parities), the tile prefix, the
// particle counts and each member's buffer parity relative to the batch's (a member
// restored from a checkpoint may sit on the other population buffer).
static cudaError_t batch_upload(ledds_batch_s* b) {
    const int n = b->nsim;
    for (int q = 0; q < 2; ++q) b->chunks[q].assign(b->nchunks, BatchChunk{});
    std::vector<LbmArgs> la(2 * n);
    std::vector<DemArgs> da(n);
    std::vector<int> ts(3 * n + 2, 0);
    bool sphd_all = true;
    for (int i = 0; i < n; ++i) {
        ledds_sim_s* s = b->sims[i];
        const int last = (s->p.n_sub - 1) & 1;
        const int off = s->parity ^ b->parity;
        la[i] = lbm_args(s, off, off ^ 1, last);
        la[n + i] = lbm_args(s, off ^ 1, off, last);
        da[i] = dem_args(s);
        ts[i + 1] = ts[i] + s->ntiles;
        sphd_all = sphd_all && !la[i].subdiv_any && !la[i].mi[0] && !la[i].mi[1] && !la[i].mi[2];
        ts[n + 1 + i] = s->P.n;
        ts[2 * n + 1 + i] = off;
    }
    // PSM work order: member order, or largest members first (their tiles are taken
    // first and the small members' tiles fill the tail of the persistent launch)
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    if (b->order == 1)
        std::stable_sort(perm.begin(), perm.end(),
                         [&](int x, int y) { return b->sims[x]->ntiles > b->sims[y]->ntiles; });
    for (int q = 0; q < 2; ++q)
        for (int c = 0; c < b->nchunks; ++c) {
            BatchChunk& ch = b->chunks[q][c];
            const int first = c * BATCH_CHUNK, cnt = std::min(BATCH_CHUNK, n - first);
            ch.nsim = cnt;
            ch.tile_start[0] = 0;
            for (int k = 0; k < cnt; ++k) {
                const int m = perm[first + k];
                ch.a[k] = la[q * n + m];
                ch.tile_start[k + 1] = ch.tile_start[k] + b->sims[m]->ntiles;
            }
        }
    CK(cudaMemcpyAsync(b->d_largs[0], la.data(), sizeof(LbmArgs) * 2 * n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_dargs, da.data(), sizeof(DemArgs) * n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_tile_start, ts.data(), sizeof(int) * (3 * n + 1), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    b->sphd = sphd_all;
    b->versions.assign(n, 0);
    for (int i = 0; i < n; ++i) b->versions[i] = b->sims[i]->version;
    return cudaSuccess;
}

static cudaError_t batch_enqueue(ledds_batch_s* b, int p, cudaStream_t st) {
    CK(cudaMemsetAsync(b->d_counter, 0, sizeof(int) * (size_t)b->nchunks, st));
    CK(launch_dem_batch(b->d_dargs, b->d_poff, b->nsim, p, st));
    CK(launch_bin_batch(b->d_largs[p], b->d_np, b->nsim, st));
    for (int c = 0; c < b->nchunks; ++c)
        CK(launch_psm_batch(b->chunks[p][c], b->d_counter + c, b->storage, b->nblocks, b->sphd, st));
    CK(launch_final_batch(b->d_dargs, b->nsim, st));
    return cudaSuccess;
}

static cudaError_t batch_capture(ledds_batch_s* b, int p, int nsteps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < nsteps && e == cudaSuccess; ++q) e = batch_enqueue(b, p ^ (q & 1), b->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    if (e2 != cudaSuccess) return e2;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

int ledds_batch_step(ledds_batch_t b, int n_steps) {
    if (!b || n_steps < 0) return LEDDS_ERR_INVALID_ARG;
    bool stale = b->versions.size() != (size_t)b->nsim;
    for (int i = 0; i < b->nsim && !stale; ++i) stale = b->versions[i] != b->sims[i]->version;
    if (stale) {
        batch_drop_graphs(b);
        if (batch_upload(b) != cudaSuccess) return LEDDS_ERR_CUDA;
    }
    int left = n_steps;
    while (left > 0) {
        const int p = b->parity;
        const int k = left >= 2 ? 2 : 1;
        cudaGraphExec_t* g = k == 2 ? &b->g2[p] : &b->g1[p];
        if (!*g && batch_capture(b, p, k, g) != cudaSuccess) return LEDDS_ERR_CUDA;
        if (cudaGraphLaunch(*g, b->stream) != cudaSuccess) return LEDDS_ERR_CUDA;
        left -= k;
        b->steps += k;
        if (k == 1) b->parity ^= 1;
        for (auto* s : b->sims) {
            s->steps += k;
            if (k == 1) s->parity ^= 1;
        }
    }
    return LEDDS_OK;
}

// Try every (resident PSM CTAs per SM, work order) and keep the fastest, timed with
// events over steps_per_trial steps after two warm-up steps per candidate (these steps
// advance the members like ledds_batch_step; every candidate computes the same step).
// Tile depth of every member: its tile counts follow (the tile lists are sized for the
// smallest depth); the uploaded arguments and the graphs are rebuilt on the next step.
static void batch_set_depth(ledds_batch_s* b, int tz) {
    b->tz = tz;
    for (auto* s : b->sims) {
        s->tz = tz;
        s->ntz = (s->d.nz + tz - 1) / tz;
        s->ntiles = s->ntx * s->nty * s->ntz;
    }
    b->versions.clear();
}

static const int kBatchDepths[3] = {8, 16, 32};

int ledds_batch_configure(ledds_batch_t b, int tile_depth, int ctas_per_sm, int order) {
    if (!b) return LEDDS_ERR_INVALID_ARG;
    if (tile_depth != 8 && tile_depth != 16 && tile_depth != 32) return LEDDS_ERR_INVALID_ARG;
    if (ctas_per_sm < 1 || ctas_per_sm > psm_batch_ctas_per_sm() || order < 0 || order > 1)
        return LEDDS_ERR_INVALID_ARG;
    batch_set_depth(b, tile_depth);
    b->ctas_per_sm = ctas_per_sm;
    b->nblocks = ctas_per_sm * b->sms;
    b->order = order;
    return LEDDS_OK;
}

int ledds_batch_get_config(ledds_batch_t b, int* tile_depth, int* ctas_per_sm, int* order) {
    if (!b || !tile_depth || !ctas_per_sm || !order) return LEDDS_ERR_INVALID_ARG;
    *tile_depth = b->tz;
    *ctas_per_sm = b->ctas_per_sm;
    *order = b->order;
    return LEDDS_OK;
}

// Choices of earlier autotuner runs, by the shape of the batch (members' dimensions and
// particle counts, storage, collision): a batch of the same shape takes the cached
// choice without trials.
static std::mutex g_tune_mu;
static std::map<unsigned long long, int> g_tune_cache;

static unsigned long long batch_shape_key(const ledds_batch_s* b) {
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](long long v) {
        for (int q = 0; q < 8; ++q) {
            h ^= (unsigned long long)((v >> (8 * q)) & 0xff);
            h *= 1099511628211ull;
        }
    };
    mix(b->nsim);
    mix(b->storage);
    mix(b->sms);
    for (const auto* s : b->sims) {
        mix(s->d.nx);
        mix(s->d.ny);
        mix(s->d.nz);
        mix(s->P.n);
        mix(s->p.collision);
    }
    return h;
}

static void batch_apply_choice(ledds_batch_s* b, int id, int max_cps) {
    const int order = id & 1, cps = (id >> 1) % max_cps + 1, d = (id >> 1) / max_cps;
    ledds_batch_configure(b, kBatchDepths[d], cps, order);
}

int ledds_batch_autotune(ledds_batch_t b, int steps_per_trial, int* choice) {
    if (!b || steps_per_trial < 1) return LEDDS_ERR_INVALID_ARG;
    const int max_cps = psm_batch_ctas_per_sm();
    const unsigned long long key = batch_shape_key(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            batch_apply_choice(b, it->second, max_cps);
            if (choice) *choice = it->second;
            return LEDDS_OK;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LEDDS_ERR_CUDA;
    float best = 0.0f;
    int best_id = -1, rc = LEDDS_OK;
    const int ncand = 3 * max_cps * 2;
    for (int id = 0; id < ncand && rc == LEDDS_OK; ++id) {
        batch_apply_choice(b, id, max_cps);
        if ((rc = ledds_batch_step(b, 2)) != LEDDS_OK) break;
        float ms = 0.0f;
        if (cudaEventRecord(e0, b->stream) != cudaSuccess) { rc = LEDDS_ERR_CUDA; break; }
        if ((rc = ledds_batch_step(b, steps_per_trial)) != LEDDS_OK) break;
        if (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = LEDDS_ERR_CUDA;
            break;
        }
        if (best_id < 0 || ms < best) {
            best = ms;
            best_id = id;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_id >= 0) {
        batch_apply_choice(b, best_id, max_cps);
        if (rc == LEDDS_OK) {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune_cache[key] = best_id;
        }
    }
    if (choice) *choice = best_id;
    return rc;
}

}  // extern "C"
