// lbm.cu -- lattice kernels of the coupled step: D3Q19 BGK collide-and-stream with
// partially saturated cells (Secs. 2.3-2.4), the solid fractions computed inside the
// collision kernel (Table 1 "Compute solid fractions"), and the per-particle reduction of
// the hydrodynamic force and torque (Eqs. forceSF, torqueSF; Table 1 "Force reduction").
//
// Layout: populations are structure-of-arrays, plane i at offset i*N, stored as
// g_i = f_i - t_i. The stored array holds post-collision values f*; a step pulls
// f_i(x) = f*_i(x - c_i) (halfway bounce-back where x - c_i is behind a wall), collides
// and writes f*(x) to the other buffer. One CTA owns a 32x8x4 tile of nodes; each warp
// processes one x-row (32 consecutive nodes: coalesced 128-byte rows for FP32). The PSM
// kernel itself is in psm.cuh; psm_aa.cu instantiates it for the single-array AA pattern,
// whose array states the read, initialisation and rebase kernels here also handle.
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include "internal.cuh"
#include "psm.cuh"

namespace ledds {


// ------------------------------------------------------------------------------------
// Pull streaming with periodic wrap and halfway bounce-back.
// ------------------------------------------------------------------------------------
struct Nbr {
    long long cell;
    int xs[3], ys[3], zs[3];   // source coordinate for c = -1, 0, +1 (index c+1)
    bool wx[3], wy[3], wz[3];  // the source lies behind a wall
};

__device__ __forceinline__ void axis_nbr(int q, int n, int per, int* s, bool* w) {
    s[1] = q;
    w[1] = false;
    int qm = q - 1, qp = q + 1;
    bool wm = false, wp = false;
    if (qm < 0) {
        if (per) qm += n;
        else { wm = true; qm = q; }
    }
    if (qp >= n) {
        if (per) qp -= n;
        else { wp = true; qp = q; }
    }
    s[2] = qm;  // c = +1: the population arrives from q - 1
    w[2] = wm;
    s[0] = qp;  // c = -1: from q + 1
    w[0] = wp;
}

__device__ __forceinline__ void make_nbr(const LbmArgs& a, int x, int y, int z, Nbr& nb) {
    nb.cell = x + (long long)a.nx * (y + (long long)a.ny * z);
    axis_nbr(x, a.nx, a.per[0], nb.xs, nb.wx);
    axis_nbr(y, a.ny, a.per[1], nb.ys, nb.wy);
    axis_nbr(z, a.nz, a.per[2], nb.zs, nb.wz);
}


// Element offset of plane i of the stored post-collision array as the two-lattice pull
// sees it: with the AA pattern after an in-place step (PSM_AA_ODD) f*_i sits in slot opp(i).
__device__ __forceinline__ long long plane(const LbmArgs& a, int i) {
    return (long long)(a.aa == PSM_AA_ODD ? OPP(i) : i) * a.N;
}

template <class SS, int I>
__device__ __forceinline__ float pull_one(const LbmArgs& a, const typename SS::T* pin,
                                          const Nbr& nb) {
    constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
    const bool wx = nb.wx[cx + 1], wy = nb.wy[cy + 1], wz = nb.wz[cz + 1];
    const bool wall = wx || wy || wz;
    long long src = nb.xs[cx + 1] + (long long)a.nx * (nb.ys[cy + 1] + (long long)a.ny * nb.zs[cz + 1]);
    long long addr = wall ? plane(a, OPP(I)) + nb.cell : plane(a, I) + src;
    float v = SS::load(pin + addr, a.inv_scale);
    if (wall) v += wall_term<I>(a.uw, wx, wy, wz);
    return v;
}

template <class SS, int I>
struct PullAll {
    static __device__ __forceinline__ void run(const LbmArgs& a, const typename SS::T* pin,
                                               const Nbr& nb, float* g) {
        g[I] = pull_one<SS, I>(a, pin, nb);
        PullAll<SS, I + 1>::run(a, pin, nb, g);
    }
};
template <class SS>
struct PullAll<SS, 19> {
    static __device__ __forceinline__ void run(const LbmArgs&, const typename SS::T*,
                                               const Nbr&, float*) {}
};

// ------------------------------------------------------------------------------------
// Initialisation: the stored array must pull back to the requested pre-collision f, so
// each value is written where the first pull will read it ("reverse streaming").
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float feq_offset(int i, float drho, float rho, float ux, float uy,
                                            float uz) {
    // f^eq_i - t_i, Eq. (equilibrium) with c_s^2 = 1/3, written around t_i.
    float cu = (float)CX(i) * ux + (float)CY(i) * uy + (float)CZ(i) * uz;
    float usq = ux * ux + uy * uy + uz * uz;
    return TW(i) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
}

template <int I>
__device__ __forceinline__ float init_one(const LbmArgs& a, const Nbr& nb, long long cell,
                                          const float* rho_in, const float* u_in, const float* f_in) {
    // The link x -> x + c_i: its far end is the node whose pull reads plane i here.
    constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
    const bool wx = nb.wx[1 - cx], wy = nb.wy[1 - cy], wz = nb.wz[1 - cz];
    const bool wall = wx || wy || wz;
    long long dst = wall ? cell
                         : nb.xs[1 - cx] + (long long)a.nx * (nb.ys[1 - cy] + (long long)a.ny * nb.zs[1 - cz]);
    constexpr int want_w = OPP(I);  // at a wall: the bounced population of x
    int want = wall ? want_w : I;
    float g;
    if (f_in) {
        g = f_in[(long long)want * a.N + dst] - (wall ? TW(want_w) : TW(I));
    } else {
        float r = rho_in ? rho_in[dst] : 1.0f;
        float ux = u_in ? u_in[dst] : 0.f, uy = u_in ? u_in[a.N + dst] : 0.f;
        float uz = u_in ? u_in[2 * a.N + dst] : 0.f;
        g = feq_offset(want, r - 1.0f, r, ux, uy, uz);
    }
    // the pull of OPP(i) at x adds its wall term; store the value that cancels it
    if (wall) g -= wall_term<OPP(I)>(a.uw, wx, wy, wz);
    return g;
}

// The AA pattern before an in-place step (PSM_AA_EVEN) holds f_i(x) itself in slot i.
__device__ __forceinline__ float init_natural(const LbmArgs& a, int i, long long cell, const float* rho_in,
                                              const float* u_in, const float* f_in) {
    if (f_in) return f_in[(long long)i * a.N + cell] - TW(i);
    float r = rho_in ? rho_in[cell] : 1.0f;
    float ux = u_in ? u_in[cell] : 0.f, uy = u_in ? u_in[a.N + cell] : 0.f;
    float uz = u_in ? u_in[2 * a.N + cell] : 0.f;
    return feq_offset(i, r - 1.0f, r, ux, uy, uz);
}

template <class SS, int I>
struct InitAll {
    static __device__ __forceinline__ void run(const LbmArgs& a, const Nbr& nb, long long cell,
                                               const float* rho, const float* u, const float* f,
                                               typename SS::T* pout) {
        if (a.aa == PSM_AA_EVEN)
            SS::store(pout + (long long)I * a.N + cell, init_natural(a, I, cell, rho, u, f), a.scale);
        else
            SS::store(pout + plane(a, I) + cell, init_one<I>(a, nb, cell, rho, u, f), a.scale);
        InitAll<SS, I + 1>::run(a, nb, cell, rho, u, f, pout);
    }
};
template <class SS>
struct InitAll<SS, 19> {
    static __device__ __forceinline__ void run(const LbmArgs&, const Nbr&, long long, const float*,
                                               const float*, const float*, typename SS::T*) {}
};

template <int STORE>
__global__ void k_init(const LbmArgs a, const float* rho_in, const float* u_in,
                       const float* f_in) {
    using SS = Store<STORE>;
    using T = typename SS::T;
    T* pout = (T*)a.pop_out;
    long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= a.N) return;
    int x = (int)(cell % a.nx);
    int y = (int)((cell / a.nx) % a.ny);
    int z = (int)(cell / ((long long)a.nx * a.ny));
    Nbr nb;
    make_nbr(a, x, y, z, nb);
    InitAll<SS, 0>::run(a, nb, cell, rho_in, u_in, f_in, pout);
}

// Changing a wall velocity keeps the current pre-collision populations: the stored
// values of wall links absorb the difference of the old and new wall terms. (The AA
// pattern before an in-place step holds the pre-collision populations themselves and
// needs no rebase.)
template <class SS, int I>
struct RebaseAll {
    static __device__ __forceinline__ void run(const LbmArgs& a, const float (&uw_old)[3][2][3],
                                               const Nbr& nb, typename SS::T* pop) {
        constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
        const bool wx = nb.wx[cx + 1], wy = nb.wy[cy + 1], wz = nb.wz[cz + 1];
        if (wx || wy || wz) {
            typename SS::T* p = pop + plane(a, OPP(I)) + nb.cell;
            float v = SS::load(p, a.inv_scale);
            v += wall_term<I>(uw_old, wx, wy, wz) - wall_term<I>(a.uw, wx, wy, wz);
            SS::store(p, v, a.scale);
        }
        RebaseAll<SS, I + 1>::run(a, uw_old, nb, pop);
    }
};
template <class SS>
struct RebaseAll<SS, 19> {
    static __device__ __forceinline__ void run(const LbmArgs&, const float (&)[3][2][3], const Nbr&,
                                               typename SS::T*) {}
};

struct WallVel {
    float uw[3][2][3];
};

template <int STORE>
__global__ void k_rebase(const LbmArgs a, const WallVel old) {
    using SS = Store<STORE>;
    long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= a.N) return;
    int x = (int)(cell % a.nx);
    int y = (int)((cell / a.nx) % a.ny);
    int z = (int)(cell / ((long long)a.nx * a.ny));
    Nbr nb;
    make_nbr(a, x, y, z, nb);
    RebaseAll<SS, 0>::run(a, old.uw, nb, (typename SS::T*)a.pop_out);
}

// f*_I(x) of the last step of the AA pattern's streaming form, from where it was pushed.
template <class SS, int I>
struct GatherPushed {
    static __device__ __forceinline__ void run(const LbmArgs& a, const typename SS::T* pop, const Nbr& nb,
                                               float* g) {
        constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
        const bool wx = nb.wx[1 - cx], wy = nb.wy[1 - cy], wz = nb.wz[1 - cz];  // x + c_I behind a wall
        if (wx || wy || wz) {
            g[I] = SS::load(pop + (long long)OPP(I) * a.N + nb.cell, a.inv_scale) -
                   wall_term<OPP(I)>(a.uw, wx, wy, wz);
        } else {
            long long dst = nb.xs[1 - cx] + (long long)a.nx * (nb.ys[1 - cy] + (long long)a.ny * nb.zs[1 - cz]);
            g[I] = SS::load(pop + (long long)I * a.N + dst, a.inv_scale);
        }
        GatherPushed<SS, I + 1>::run(a, pop, nb, g);
    }
};
template <class SS>
struct GatherPushed<SS, 19> {
    static __device__ __forceinline__ void run(const LbmArgs&, const typename SS::T*, const Nbr&, float*) {}
};

// Read back: pre-collision populations (which = 0) or the stored post-collision array
// (which = 1) as f, or the moments rho and u (Eqs. rho, momentum).
template <int STORE>
__global__ void k_read(const LbmArgs a, float* rho_out, float* u_out, float* f_out, int which) {
    using SS = Store<STORE>;
    using T = typename SS::T;
    const T* pin = (const T*)a.pop_in;
    long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= a.N) return;
    float g[19];
    if (a.aa == PSM_AA_EVEN) {
        // the array holds the pre-collision f; the last step's f*_i(x) went to x + c_i
        // (or, for a link into a wall, came back to x with the wall term of opp(i))
        if (which == 1) {
            int x = (int)(cell % a.nx);
            int y = (int)((cell / a.nx) % a.ny);
            int z = (int)(cell / ((long long)a.nx * a.ny));
            Nbr nb;
            make_nbr(a, x, y, z, nb);
            GatherPushed<SS, 0>::run(a, pin, nb, g);
        } else {
#pragma unroll
            for (int i = 0; i < 19; ++i) g[i] = SS::load(pin + (long long)i * a.N + cell, a.inv_scale);
        }
    } else if (which == 1) {
#pragma unroll
        for (int i = 0; i < 19; ++i) g[i] = SS::load(pin + plane(a, i) + cell, a.inv_scale);
    } else {
        int x = (int)(cell % a.nx);
        int y = (int)((cell / a.nx) % a.ny);
        int z = (int)(cell / ((long long)a.nx * a.ny));
        Nbr nb;
        make_nbr(a, x, y, z, nb);
        PullAll<SS, 0>::run(a, pin, nb, g);
    }
    if (f_out) {
#pragma unroll
        for (int i = 0; i < 19; ++i) f_out[(long long)i * a.N + cell] = g[i] + TW(i);
    }
    if (rho_out || u_out) {
        float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            drho += g[i];
            jx += (float)CX(i) * g[i];
            jy += (float)CY(i) * g[i];
            jz += (float)CZ(i) * g[i];
        }
        float rho = 1.0f + drho;
        if (a.has_force) {
            jx += 0.5f * a.F[0];
            jy += 0.5f * a.F[1];
            jz += 0.5f * a.F[2];
        }
        if (rho_out) rho_out[cell] = rho;
        if (u_out) {
            u_out[cell] = jx / rho;
            u_out[a.N + cell] = jy / rho;
            u_out[2 * a.N + cell] = jz / rho;
        }
    }
}

// ------------------------------------------------------------------------------------
// Tile binning: every particle appends its id to the lists of the tiles its solid
// fraction can reach (node range r +- reach, periodic wrap).
// ------------------------------------------------------------------------------------

// The tiles (of T nodes) along one axis that the node range [ceil(r - reach),
// floor(r + reach)] meets, clipped to the lattice or wrapped on a periodic axis: one or two
// contiguous runs s0 .. s0 + n0 - 1 and s1 .. s1 + n1 - 1, at most 16 tiles in all.
struct AxisRuns {
    int s0, n0, s1, n1;
    __device__ int count() const { return n0 + n1; }
    __device__ int tile(int m) const { return m < n0 ? s0 + m : s1 + (m - n0); }
};

__device__ __forceinline__ AxisRuns axis_runs(double r, float reach, int n, int per, int T) {
    AxisRuns R{0, 0, 0, 0};
    // a particle far outside the lattice (or not finite) reaches no tile
    if (!(r > -2.0 * n && r < 3.0 * n)) return R;
    int lo = (int)ceil(r - (double)reach);
    int hi = (int)floor(r + (double)reach);
    if (lo > hi) return R;  // no node within reach
    const int nt = (n + T - 1) / T;
    int t0 = 0, t1 = -1, u0 = 0, u1 = -1;  // runs [t0, t1] and [u0, u1]
    if (!per) {
        lo = max(lo, 0);
        hi = min(hi, n - 1);
        if (lo <= hi) {
            t0 = lo / T;
            t1 = hi / T;
        }
    } else if (hi - lo + 1 >= n) {
        t1 = nt - 1;
    } else {
        int lw = lo % n;
        if (lw < 0) lw += n;
        const int hw = lw + (hi - lo);
        if (hw < n) {
            t0 = lw / T;
            t1 = hw / T;
        } else {
            const int a0 = lw / T, b1 = (hw - n) / T;  // [a0, nt - 1] and [0, b1]
            if (b1 >= a0) {
                t1 = nt - 1;  // the two runs meet: every tile
            } else {
                t0 = a0;
                t1 = nt - 1;
                u1 = b1;
            }
        }
    }
    R.s0 = t0;
    R.n0 = min(16, max(0, t1 - t0 + 1));
    R.s1 = u0;
    R.n1 = min(16 - R.n0, max(0, u1 - u0 + 1));
    return R;
}

__device__ __forceinline__ int axis_tiles(double r, float reach, int n, int per, int T, int* out) {
    const AxisRuns R = axis_runs(r, reach, n, per, T);
    for (int m = 0; m < R.count(); ++m) out[m] = R.tile(m);
    return R.count();
}

// One warp per particle: the lanes append its id to the tiles' lists in parallel.
__global__ void k_bin(const LbmArgs a, int n, int* tile_count, int* tile_ids) {
    const int k = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= n) return;  // uniform across the warp
    double r[3] = {a.st[(SP + 0) * a.pcap + k], a.st[(SP + 1) * a.pcap + k],
                   a.st[(SP + 2) * a.pcap + k]};
    float reach = reach_of(a, a.shape[k], a.radius[k], a.bound[k]);
    if (!(isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]))) {
        if (lane == 0) atomicAdd(&a.status->nan_detected, 1);
        return;
    }
    const AxisRuns X = axis_runs(r[0], reach, a.nx, a.per[0], TILE_X);
    const AxisRuns Y = axis_runs(r[1], reach, a.ny, a.per[1], TILE_Y);
    const AxisRuns Z = axis_runs(r[2], reach, a.nz, a.per[2], a.tz);
    const int cx = X.count(), n01 = cx * Y.count(), total = n01 * Z.count();
    for (int m = lane; m < total; m += 32) {
        const int c = m / n01, rem = m - c * n01, b = rem / cx, q = rem - b * cx;
        const int t = (Z.tile(c) * a.nty + Y.tile(b)) * a.ntx + X.tile(q);
        const int slot = atomicAdd(&tile_count[t], 1);
        if (slot < a.tile_cap) tile_ids[(long long)t * a.tile_cap + slot] = k;
        else atomicAdd(&a.status->tile_overflow, 1);
    }
}


// Batched form: persistent CTAs take (simulation, tile) work items from a queue, so many
// simulations of uneven sizes advance in one launch with balanced load. The members'
// arguments travel in the launch's parameter block (read-only for the whole launch, like
// the single-simulation kernel's argument), up to BATCH_CHUNK members per launch.
// The batched kernel indexes its members' arguments at run time and runs best with the
// larger register budget (2 resident CTAs per SM) for every storage format. Tiles are
// TILE_X x TILE_Y x tz nodes, tz chosen per batch (ledds_batch_configure / autotune).
// SPHD: every member's particles are spheres with distance fractions and no offset needs
// a periodic wrap.
constexpr int PSM_BATCH_MINB = 2;

template <int STORE, bool TRT, bool SPHD>
__global__ void __launch_bounds__(PSM_THREADS, PSM_BATCH_MINB) k_psm_batch(const __grid_constant__ BatchChunk P,
                                                                          int* counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item, s_sim;
    const int nsim = P.nsim;
    const int total = P.tile_start[nsim];
    for (;;) {
        if (threadIdx.x == 0) {
            int item = atomicAdd(counter, 1);
            int lo = 0, hi = nsim - 1;
            while (lo < hi) {  // last simulation whose first tile is <= item
                int mid = (lo + hi + 1) >> 1;
                if (P.tile_start[mid] <= item) lo = mid;
                else hi = mid - 1;
            }
            s_item = item;
            s_sim = lo;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int sim = s_sim;
        const LbmArgs& a = P.a[sim];
        const int t = item - P.tile_start[sim];
        const int bx = t % a.ntx, by = (t / a.ntx) % a.nty, bz = t / (a.ntx * a.nty);
        psm_tile_direct<STORE, TRT, PSM_AB, SPHD>(a, bx, by, bz, 0, a.tz, smem);
        __syncthreads();
    }
}

// Tile binning of every simulation of a batch: one CTA per simulation clears its tile
// lists and hydrodynamic sums, then bins its particles.
__device__ __forceinline__ void bin_particle(const LbmArgs& a, int k, int* tile_count, int* tile_ids) {
    double r[3] = {a.st[(SP + 0) * a.pcap + k], a.st[(SP + 1) * a.pcap + k], a.st[(SP + 2) * a.pcap + k]};
    float reach = reach_of(a, a.shape[k], a.radius[k], a.bound[k]);
    if (!(isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]))) {
        atomicAdd(&a.status->nan_detected, 1);
        return;
    }
    int tl[3][16], tcn[3];
    tcn[0] = axis_tiles(r[0], reach, a.nx, a.per[0], TILE_X, tl[0]);
    tcn[1] = axis_tiles(r[1], reach, a.ny, a.per[1], TILE_Y, tl[1]);
    tcn[2] = axis_tiles(r[2], reach, a.nz, a.per[2], a.tz, tl[2]);
    for (int c = 0; c < tcn[2]; ++c)
        for (int b = 0; b < tcn[1]; ++b)
            for (int q = 0; q < tcn[0]; ++q) {
                int t = (tl[2][c] * a.nty + tl[1][b]) * a.ntx + tl[0][q];
                int slot = atomicAdd(&tile_count[t], 1);
                if (slot < a.tile_cap) tile_ids[(long long)t * a.tile_cap + slot] = k;
                else atomicAdd(&a.status->tile_overflow, 1);
            }
}

__global__ void k_bin_batch(const LbmArgs* args, const int* np) {
    const LbmArgs& a = args[blockIdx.x];
    const int n = np[blockIdx.x];
    int* tcount = const_cast<int*>(a.tile_count);
    int* tids = const_cast<int*>(a.tile_ids);
    const int ntiles = a.ntx * a.nty * a.ntz;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) tcount[t] = 0;
    for (int i = threadIdx.x; i < 3 * a.pcap; i += blockDim.x) {
        a.Fh[i] = 0.0;
        a.Mh[i] = 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) bin_particle(a, k, tcount, tids);
}

int psm_batch_ctas_per_sm() { return PSM_BATCH_MINB; }

// Tensor maps of a population array for the staged PSM route: 4D (x, y, z, plane), boxes
// of TILE_Y rows by TILE_X columns (narrow) or TILE_X + 2H columns (wide, H = 16 bytes of
// elements), one plane deep; elements outside the array read as zero. False when the
// lattice does not suit the route (rows not a multiple of 16 bytes, fewer rows than a
// tile, narrower than a wide box) or the driver has no tensor-map encoder; the kernel
// then takes the direct route.
bool psm_make_maps(const void* pop, int store, int nx, int ny, int nz, PsmMaps* out) {
    const int es = (int)storage_bytes(store);
    const int H = 16 / es;
    if (((long long)nx * es) % 16 != 0 || (reinterpret_cast<uintptr_t>(pop) & 15u) != 0) return false;
    if (nx < TILE_X + 2 * H || ny < TILE_Y || nz < 1) return false;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, 19};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * es, (cuuint64_t)nx * ny * es, (cuuint64_t)nx * ny * nz * es};
    const cuuint32_t box_n[4] = {TILE_X, TILE_Y, 1, 1};
    const cuuint32_t box_w[4] = {(cuuint32_t)(TILE_X + 2 * H), TILE_Y, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    PsmMaps m;
    memset(&m, 0, sizeof(m));
    if (encode(&m.narrow, dt, 4, const_cast<void*>(pop), dims, strides, box_n, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (encode(&m.wide, dt, 4, const_cast<void*>(pop), dims, strides, box_w, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    *out = m;
    return true;
}

// Solid fractions only (the same tile machinery), for inspection.
__global__ void __launch_bounds__(256) k_voxelize(const LbmArgs a, float* beta, int* ids, int* nsolid) {
    __shared__ TileCache tc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = blockIdx.x * TILE_X, y0 = blockIdx.y * TILE_Y, z0 = blockIdx.z * a.tz;
    const int tile = (blockIdx.z * a.nty + blockIdx.y) * a.ntx + blockIdx.x;
    const int cnt = min(a.tile_count[tile], a.tile_cap);
    load_tile(a, tc, tile, cnt, x0, y0, z0);
    __syncthreads();
    const int x = x0 + lane, y = y0 + warp;
    for (int iz = 0; iz < a.tz; ++iz) {
        const int z = z0 + iz;
        if (y >= a.ny || z >= a.nz) break;
        const unsigned long long mask = cnt ? row_mask<true>(a, tc, cnt, warp, iz) : 0ull;
        const bool valid = x < a.nx;
        Two t;
        t.ns = 0;
        t.total = 0;
        if (mask) node_solids<false>(a, tc, mask, lane, warp, iz, x, y, z, valid, t);  // uniform
        if (!valid) continue;
        long long cell = x + (long long)a.nx * (y + (long long)a.ny * z);
        beta[2 * cell] = t.ns > 0 ? t.b0 : 0.f;
        beta[2 * cell + 1] = t.ns > 1 ? t.b1 : 0.f;
        ids[2 * cell] = t.ns > 0 ? tc_pid(tc, t.e0) : -1;
        ids[2 * cell + 1] = t.ns > 1 ? tc_pid(tc, t.e1) : -1;
        nsolid[cell] = t.total;
    }
}

// ------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------
static dim3 tile_grid(const LbmArgs& a) { return dim3(a.ntx, a.nty, a.ntz); }

cudaError_t launch_init(const LbmArgs& a, int store, const float* rho, const float* u,
                        const float* f, cudaStream_t s) {
    unsigned blocks = (unsigned)((a.N + 255) / 256);
    if (store == LEDDS_STORE_F32) k_init<LEDDS_STORE_F32><<<blocks, 256, 0, s>>>(a, rho, u, f);
    else if (store == LEDDS_STORE_F16) k_init<LEDDS_STORE_F16><<<blocks, 256, 0, s>>>(a, rho, u, f);
    else k_init<LEDDS_STORE_BF16><<<blocks, 256, 0, s>>>(a, rho, u, f);
    return cudaGetLastError();
}

cudaError_t launch_rebase(const LbmArgs& a, int store, const float (*uw_old)[2][3], cudaStream_t s) {
    unsigned blocks = (unsigned)((a.N + 255) / 256);
    WallVel w;
    for (int q = 0; q < 3; ++q)
        for (int e = 0; e < 2; ++e)
            for (int c = 0; c < 3; ++c) w.uw[q][e][c] = uw_old[q][e][c];
    if (store == LEDDS_STORE_F32) k_rebase<LEDDS_STORE_F32><<<blocks, 256, 0, s>>>(a, w);
    else if (store == LEDDS_STORE_F16) k_rebase<LEDDS_STORE_F16><<<blocks, 256, 0, s>>>(a, w);
    else k_rebase<LEDDS_STORE_BF16><<<blocks, 256, 0, s>>>(a, w);
    return cudaGetLastError();
}

cudaError_t launch_read(const LbmArgs& a, int store, float* rho, float* u, float* f, int which,
                        cudaStream_t s) {
    unsigned blocks = (unsigned)((a.N + 255) / 256);
    if (store == LEDDS_STORE_F32) k_read<LEDDS_STORE_F32><<<blocks, 256, 0, s>>>(a, rho, u, f, which);
    else if (store == LEDDS_STORE_F16) k_read<LEDDS_STORE_F16><<<blocks, 256, 0, s>>>(a, rho, u, f, which);
    else k_read<LEDDS_STORE_BF16><<<blocks, 256, 0, s>>>(a, rho, u, f, which);
    return cudaGetLastError();
}

cudaError_t launch_bin(const LbmArgs& a, int n, int* tile_count, int* tile_ids, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_bin<<<(unsigned)(((long long)n * 32 + 127) / 128), 128, 0, s>>>(a, n, tile_count, tile_ids);
    return cudaGetLastError();
}

cudaError_t launch_psm(const LbmArgs& a, const PsmMaps* m, int store, cudaStream_t s) {
    if (a.w64) return launch_psm_wide(a, m, store, s);
    if (a.aa != PSM_AB) return launch_psm_aa(a, m, store, s);
    return launch_psm_mode<PSM_AB>(a, m, store, s);
}

template <int STORE, bool TRT, bool SPHD>
static cudaError_t launch_psm_batch_t(const BatchChunk& P, int* counter, int nblocks, cudaStream_t s) {
    static bool configured = false;
    const size_t smem = PsmSmem<STORE, false, true>::bytes;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_psm_batch<STORE, TRT, SPHD>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_psm_batch<STORE, TRT, SPHD><<<nblocks, PSM_THREADS, smem, s>>>(P, counter);
    return cudaGetLastError();
}

template <bool SPHD>
static cudaError_t launch_psm_batch_g(const BatchChunk& P, int* counter, int store, int nblocks, cudaStream_t s) {
    if (P.a[0].trt) {
        if (store == LEDDS_STORE_F32) return launch_psm_batch_t<LEDDS_STORE_F32, true, SPHD>(P, counter, nblocks, s);
        if (store == LEDDS_STORE_F16) return launch_psm_batch_t<LEDDS_STORE_F16, true, SPHD>(P, counter, nblocks, s);
        return launch_psm_batch_t<LEDDS_STORE_BF16, true, SPHD>(P, counter, nblocks, s);
    }
    if (store == LEDDS_STORE_F32) return launch_psm_batch_t<LEDDS_STORE_F32, false, SPHD>(P, counter, nblocks, s);
    if (store == LEDDS_STORE_F16) return launch_psm_batch_t<LEDDS_STORE_F16, false, SPHD>(P, counter, nblocks, s);
    return launch_psm_batch_t<LEDDS_STORE_BF16, false, SPHD>(P, counter, nblocks, s);
}

// All members of a batch share the storage format and the collision operator; sphd when
// every member qualifies for the sphere-distance form.
cudaError_t launch_psm_batch(const BatchChunk& P, int* counter, int store, int nblocks, bool sphd, cudaStream_t s) {
    if (sphd) return launch_psm_batch_g<true>(P, counter, store, nblocks, s);
    return launch_psm_batch_g<false>(P, counter, store, nblocks, s);
}

cudaError_t launch_bin_batch(const LbmArgs* args, const int* np, int nsim, cudaStream_t s) {
    k_bin_batch<<<nsim, 256, 0, s>>>(args, np);
    return cudaGetLastError();
}

cudaError_t launch_voxelize(const LbmArgs& a, float* beta, int* ids, int* nsolid, cudaStream_t s) {
    k_voxelize<<<tile_grid(a), 256, 0, s>>>(a, beta, ids, nsolid);
    return cudaGetLastError();
}

}  // namespace ledds
