// lbm.cu -- lattice kernels of the coupled step: D3Q19 BGK collide-and-stream with
// partially saturated cells (Secs. 2.3-2.4), the solid fractions computed inside the
// collision kernel (Table 1 "Compute solid fractions"), and the per-particle reduction of
// the hydrodynamic force and torque (Eqs. forceSF, torqueSF; Table 1 "Force reduction").
//
// Layout: populations are structure-of-arrays, plane i at offset i*N, stored as
// g_i = f_i - t_i. The stored array holds post-collision values f*; a step pulls
// f_i(x) = f*_i(x - c_i) (halfway bounce-back where x - c_i is behind a wall), collides
// and writes f*(x) to the other buffer. One CTA owns a 32x8x4 tile of nodes; each warp
// processes one x-row (32 consecutive nodes: coalesced 128-byte rows for FP32).
#include <math.h>
#include <string.h>

#include "internal.cuh"

namespace ledds {

constexpr unsigned FULL = 0xffffffffu;

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

// Moving-wall correction 6 t_i (c_i . u_w) (rho_w = 1) for a link that crossed walls;
// with walls on two axes the wall of the higher axis (z, then y, then x) is used. The
// side of each axis is fixed by the sign of c_i, so every parameter index is constant.
template <int I>
__device__ __forceinline__ float wall_term(const float (&uw)[3][2][3], bool wx, bool wy, bool wz) {
    constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
    constexpr int sx = cx == 1 ? 0 : 1, sy = cy == 1 ? 0 : 1, sz = cz == 1 ? 0 : 1;
    float u0 = wz ? uw[2][sz][0] : (wy ? uw[1][sy][0] : uw[0][sx][0]);
    float u1 = wz ? uw[2][sz][1] : (wy ? uw[1][sy][1] : uw[0][sx][1]);
    float u2 = wz ? uw[2][sz][2] : (wy ? uw[1][sy][2] : uw[0][sx][2]);
    return 6.0f * TW(I) * ((float)cx * u0 + (float)cy * u1 + (float)cz * u2);
}

template <class SS, int I>
__device__ __forceinline__ float pull_one(const LbmArgs& a, const typename SS::T* pin,
                                          const Nbr& nb) {
    constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
    const bool wx = nb.wx[cx + 1], wy = nb.wy[cy + 1], wz = nb.wz[cz + 1];
    const bool wall = wx || wy || wz;
    long long src = nb.xs[cx + 1] + (long long)a.nx * (nb.ys[cy + 1] + (long long)a.ny * nb.zs[cz + 1]);
    long long addr = wall ? (long long)OPP(I) * a.N + nb.cell : (long long)I * a.N + src;
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

template <class SS, int I>
struct InitAll {
    static __device__ __forceinline__ void run(const LbmArgs& a, const Nbr& nb, long long cell,
                                               const float* rho, const float* u, const float* f,
                                               typename SS::T* pout) {
        SS::store(pout + (long long)I * a.N + cell, init_one<I>(a, nb, cell, rho, u, f), a.scale);
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
// values of wall links absorb the difference of the old and new wall terms.
template <class SS, int I>
struct RebaseAll {
    static __device__ __forceinline__ void run(const LbmArgs& a, const float (&uw_old)[3][2][3],
                                               const Nbr& nb, typename SS::T* pop) {
        constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
        const bool wx = nb.wx[cx + 1], wy = nb.wy[cy + 1], wz = nb.wz[cz + 1];
        if (wx || wy || wz) {
            typename SS::T* p = pop + (long long)OPP(I) * a.N + nb.cell;
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
    if (which == 1) {
#pragma unroll
        for (int i = 0; i < 19; ++i) g[i] = SS::load(pin + (long long)i * a.N + cell, a.inv_scale);
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
__device__ __forceinline__ float reach_of(const LbmArgs& a, int shape, double R, double Rb) {
    // distance method: beta > 0 iff |x - r| < R + R_c; subdivision: samples lie within
    // 0.78 of the node, use the bounding radius plus the cell half-diagonal.
    if (shape == LEDDS_SPHERE && a.voxel == LEDDS_VOXEL_DISTANCE) return (float)R + a.Rc + 1e-3f;
    return (float)Rb + 0.8661f + 1e-3f;
}

__device__ __forceinline__ int axis_tiles(double r, float reach, int n, int per, int T, int* out) {
    int lo = (int)ceil(r - (double)reach);
    int hi = (int)floor(r + (double)reach);
    int cnt = 0, last = -1;
    for (int q = lo; q <= hi; ++q) {
        int qw = q;
        if (per) {
            qw %= n;
            if (qw < 0) qw += n;
        } else if (q < 0 || q >= n) {
            continue;
        }
        int t = qw / T;
        if (t != last && cnt < 16) {
            bool dup = false;
            for (int m = 0; m < cnt; ++m) dup |= (out[m] == t);
            if (!dup) out[cnt++] = t;
            last = t;
        }
    }
    return cnt;
}

__global__ void k_bin(const LbmArgs a, int n, int* tile_count, int* tile_ids) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double r[3] = {a.st[(SP + 0) * a.pcap + k], a.st[(SP + 1) * a.pcap + k],
                   a.st[(SP + 2) * a.pcap + k]};
    float reach = reach_of(a, a.shape[k], a.radius[k], a.bound[k]);
    int tl[3][16], tc[3];
    tc[0] = axis_tiles(r[0], reach, a.nx, a.per[0], TILE_X, tl[0]);
    tc[1] = axis_tiles(r[1], reach, a.ny, a.per[1], TILE_Y, tl[1]);
    tc[2] = axis_tiles(r[2], reach, a.nz, a.per[2], TILE_Z, tl[2]);
    for (int c = 0; c < tc[2]; ++c)
        for (int b = 0; b < tc[1]; ++b)
            for (int q = 0; q < tc[0]; ++q) {
                int t = (tl[2][c] * a.nty + tl[1][b]) * a.ntx + tl[0][q];
                int slot = atomicAdd(&tile_count[t], 1);
                if (slot < a.tile_cap) tile_ids[(long long)t * a.tile_cap + slot] = k;
                else atomicAdd(&a.status->tile_overflow, 1);
            }
}

// ------------------------------------------------------------------------------------
// Per-tile particle cache and solid fractions (Sec. 2.4)
// ------------------------------------------------------------------------------------
struct TileCache {
    float r[3][MAX_TILE_CAP];     // centre minus tile origin (FP32, minimum image)
    double p[3][MAX_TILE_CAP];    // centre (FP64) for the exact subdivision path
    float R[MAX_TILE_CAP];        // radius (spheres) / bounding radius (ellipsoids)
    float R2[MAX_TILE_CAP];       // fl32(R*R) of the subdivision predicate
    float reach2[MAX_TILE_CAP];
    float v[3][MAX_TILE_CAP];
    float w[3][MAX_TILE_CAP];
    float m[9][MAX_TILE_CAP];     // ellipsoid rows fl32(d_j / semi_j)
    int pid[MAX_TILE_CAP];
    int shape[MAX_TILE_CAP];
    double acc[6][MAX_TILE_CAP];  // force and torque sums of this tile
};

__device__ __forceinline__ double min_image_d(double d, int per, double L) {
    if (per) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}
__device__ __forceinline__ float min_image_f(float d, int per, float L) {
    if (per) {
        if (d > 0.5f * L) d -= L;
        else if (d < -0.5f * L) d += L;
    }
    return d;
}

__device__ void load_tile(const LbmArgs& a, TileCache& tc, int tile, int cnt, int x0, int y0,
                          int z0) {
    const double org[3] = {(double)x0, (double)y0, (double)z0};
    const double Ls[3] = {(double)a.nx, (double)a.ny, (double)a.nz};
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int k = a.tile_ids[(long long)tile * a.tile_cap + e];
        tc.pid[e] = k;
        int sh = a.shape[k];
        tc.shape[e] = sh;
        for (int c = 0; c < 3; ++c) {
            double pc = a.st[(SP + c) * a.pcap + k];
            tc.p[c][e] = pc;
            tc.r[c][e] = (float)min_image_d(pc - org[c], a.per[c], Ls[c]);
            tc.v[c][e] = (float)a.st[(SV + c) * a.pcap + k];
            tc.w[c][e] = (float)a.st[(SW + c) * a.pcap + k];
        }
        double R = sh == LEDDS_SPHERE ? a.radius[k] : a.bound[k];
        tc.R[e] = (float)R;
        tc.R2[e] = __double2float_rn(R * R);
        float reach = reach_of(a, sh, a.radius[k], a.bound[k]);
        tc.reach2[e] = reach * reach;
        if (sh == LEDDS_ELLIPSOID) {
            for (int j = 0; j < 3; ++j)
                for (int c = 0; c < 3; ++c)
                    tc.m[3 * j + c][e] = __double2float_rn(
                        a.st[(ST + 3 * j + c) * a.pcap + k] / a.semi[j * a.pcap + k]);
        }
        for (int c = 0; c < 6; ++c) tc.acc[c][e] = 0.0;
    }
}

// Subdivision count: n^3 sample points (2m+1-n)/(2n) around the node, strictly inside
// the solid. FP32 with explicit round-to-nearest intrinsics (no contraction), in the
// evaluation order documented for the method, so counts are exact integers. Kept out of
// line: it runs only for nodes the exact early-outs cannot decide.
__device__ __noinline__ int subdiv_count(const TileCache& tc, int e, float px, float py, float pz,
                                         int n) {
    float o[16];
    for (int q = 0; q < n; ++q) o[q] = __fdiv_rn((float)(2 * q + 1 - n), (float)(2 * n));
    int count = 0;
    if (tc.shape[e] == LEDDS_SPHERE) {
        const float R2 = tc.R2[e];
        for (int i = 0; i < n; ++i) {
            float dx = __fadd_rn(px, o[i]);
            float xx = __fmul_rn(dx, dx);
            for (int j = 0; j < n; ++j) {
                float dy = __fadd_rn(py, o[j]);
                float s01 = __fadd_rn(xx, __fmul_rn(dy, dy));
                for (int q = 0; q < n; ++q) {
                    float dz = __fadd_rn(pz, o[q]);
                    count += __fadd_rn(s01, __fmul_rn(dz, dz)) < R2;
                }
            }
        }
    } else {
        float mm[9];
        for (int q = 0; q < 9; ++q) mm[q] = tc.m[q][e];
        for (int i = 0; i < n; ++i) {
            float dx = __fadd_rn(px, o[i]);
            float a0 = __fmul_rn(mm[0], dx), a1 = __fmul_rn(mm[3], dx), a2 = __fmul_rn(mm[6], dx);
            for (int j = 0; j < n; ++j) {
                float dy = __fadd_rn(py, o[j]);
                float t0 = __fadd_rn(a0, __fmul_rn(mm[1], dy));
                float t1 = __fadd_rn(a1, __fmul_rn(mm[4], dy));
                float t2 = __fadd_rn(a2, __fmul_rn(mm[7], dy));
                for (int q = 0; q < n; ++q) {
                    float dz = __fadd_rn(pz, o[q]);
                    float q0 = __fadd_rn(t0, __fmul_rn(mm[2], dz));
                    float q1 = __fadd_rn(t1, __fmul_rn(mm[5], dz));
                    float q2 = __fadd_rn(t2, __fmul_rn(mm[8], dz));
                    float s = __fadd_rn(__fadd_rn(__fmul_rn(q0, q0), __fmul_rn(q1, q1)), __fmul_rn(q2, q2));
                    count += s < 1.0f;
                }
            }
        }
    }
    return count;
}

// Exact subdivision path: node minus centre in FP64 (minimum image), rounded to FP32.
__device__ __noinline__ float beta_subdiv_exact(const LbmArgs& a, const TileCache& tc, int e, int x,
                                                int y, int z) {
    const int n = a.subdiv_n;
    float px = __double2float_rn(min_image_d((double)x - tc.p[0][e], a.per[0], (double)a.nx));
    float py = __double2float_rn(min_image_d((double)y - tc.p[1][e], a.per[1], (double)a.ny));
    float pz = __double2float_rn(min_image_d((double)z - tc.p[2][e], a.per[2], (double)a.nz));
    int cnt = subdiv_count(tc, e, px, py, pz, n);
    return (float)cnt / (float)(n * n * n);
}

// Solid fraction of cached particle e at node (x,y,z); (dx,dy,dz) = node - centre (FP32).
__device__ __forceinline__ float beta_of(const LbmArgs& a, const TileCache& tc, int e, int x, int y,
                                         int z, float dx, float dy, float dz) {
    const int sh = tc.shape[e];
    const float d2 = dx * dx + dy * dy + dz * dz;
    if (sh == LEDDS_SPHERE && a.voxel == LEDDS_VOXEL_DISTANCE) {
        // Eq. (naiveSolidFrac)
        float dsc = tc.R[e] + a.Rc - sqrtf(d2);
        return fminf(fmaxf(dsc / (2.0f * a.Rc), 0.0f), 1.0f);
    }
    const int n = a.subdiv_n;
    const float h = (float)(n - 1) / (float)(2 * n);  // largest sample offset
    const float hd = 1.7320508f * h;                  // sample-to-node distance bound
    // exact early-outs (margins far above FP32 rounding): no sample can be inside ...
    const float far = tc.R[e] + hd + 1e-3f;
    if (d2 > far * far) return 0.0f;
    if (sh == LEDDS_SPHERE) {
        const float nearr = tc.R[e] - hd - 1e-3f;
        if (nearr > 0.0f && d2 < nearr * nearr) return 1.0f;  // ... or every sample is
    } else {
        // every corner of the sample box strictly inside (convexity) => all samples are
        bool all_in = true;
#pragma unroll
        for (int cnr = 0; cnr < 8; ++cnr) {
            float px = dx + ((cnr & 1) ? h : -h);
            float py = dy + ((cnr & 2) ? h : -h);
            float pz = dz + ((cnr & 4) ? h : -h);
            float q0 = tc.m[0][e] * px + tc.m[1][e] * py + tc.m[2][e] * pz;
            float q1 = tc.m[3][e] * px + tc.m[4][e] * py + tc.m[5][e] * pz;
            float q2 = tc.m[6][e] * px + tc.m[7][e] * py + tc.m[8][e] * pz;
            all_in = all_in && (q0 * q0 + q1 * q1 + q2 * q2 < 0.999f);
        }
        if (all_in) return 1.0f;
    }
    return beta_subdiv_exact(a, tc, e, x, y, z);
}

// Row prefilter: which cached particles can touch the x-row (ly, lz) of this tile.
__device__ __forceinline__ unsigned long long row_mask(const LbmArgs& a, const TileCache& tc,
                                                       int cnt, int ly, int lz) {
    const int lane = threadIdx.x & 31;
    unsigned long long mask = 0ull;
    for (int base = 0; base < cnt; base += 32) {
        int e = base + lane;
        bool hit = false;
        if (e < cnt) {
            float dy = min_image_f((float)ly - tc.r[1][e], a.per[1], (float)a.ny);
            float dz = min_image_f((float)lz - tc.r[2][e], a.per[2], (float)a.nz);
            hit = dy * dy + dz * dz < tc.reach2[e];
        }
        unsigned b = __ballot_sync(FULL, hit);
        mask |= (unsigned long long)b << base;
    }
    return mask;
}

// Up to two solids per node (Sec. 3.2.3): keep the two largest beta, ties to the lower
// particle id; `total` counts every solid with beta > 0. Everything stays in registers.
struct Two {
    int ns, total;
    int e0, e1;
    float b0, b1;
};

__device__ __forceinline__ bool ranks_before(const TileCache& tc, float b, int e, float bw, int ew) {
    return b > bw || (b == bw && tc.pid[e] < tc.pid[ew]);
}

__device__ __forceinline__ void node_solids(const LbmArgs& a, const TileCache& tc,
                                            unsigned long long mask, int lx, int ly, int lz, int x,
                                            int y, int z, Two& t) {
    t.ns = 0;
    t.total = 0;
    t.e0 = t.e1 = 0;
    t.b0 = t.b1 = 0.f;
    while (mask) {
        const int e = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        float dx = min_image_f((float)lx - tc.r[0][e], a.per[0], (float)a.nx);
        float dy = min_image_f((float)ly - tc.r[1][e], a.per[1], (float)a.ny);
        float dz = min_image_f((float)lz - tc.r[2][e], a.per[2], (float)a.nz);
        float b = beta_of(a, tc, e, x, y, z, dx, dy, dz);
        if (!(b > 0.0f)) continue;
        t.total++;
        if (t.ns == 0) {
            t.e0 = e; t.b0 = b; t.ns = 1;
        } else if (ranks_before(tc, b, e, t.b0, t.e0)) {
            t.e1 = t.e0; t.b1 = t.b0; t.e0 = e; t.b0 = b; t.ns = 2;
        } else if (t.ns == 1 || ranks_before(tc, b, e, t.b1, t.e1)) {
            t.e1 = e; t.b1 = b; t.ns = 2;
        }
    }
}

// One solid's data at a node: B_k (Eq. bk), surface velocity u_k = v_k + w_k x (x - r_k),
// the arm x - r_k, and the running sum of Omega^s_{i,k} c_i.
struct SolidAt {
    float B, ux, uy, uz, usq, ax, ay, az, sx, sy, sz;
};

__device__ __forceinline__ void solid_at(const LbmArgs& a, const TileCache& tc, int e, float b, int lx,
                                         int ly, int lz, float tau, SolidAt& q) {
    q.ax = min_image_f((float)lx - tc.r[0][e], a.per[0], (float)a.nx);
    q.ay = min_image_f((float)ly - tc.r[1][e], a.per[1], (float)a.ny);
    q.az = min_image_f((float)lz - tc.r[2][e], a.per[2], (float)a.nz);
    q.B = b * (tau - 0.5f) / ((1.0f - b) + (tau - 0.5f));
    q.ux = tc.v[0][e] + (tc.w[1][e] * q.az - tc.w[2][e] * q.ay);
    q.uy = tc.v[1][e] + (tc.w[2][e] * q.ax - tc.w[0][e] * q.az);
    q.uz = tc.v[2][e] + (tc.w[0][e] * q.ay - tc.w[1][e] * q.ax);
    q.usq = q.ux * q.ux + q.uy * q.uy + q.uz * q.uz;
    q.sx = q.sy = q.sz = 0.f;
}

// Warp reduction of one solid slot's force and torque into the tile accumulators:
// one butterfly per distinct cached particle present in the warp.
__device__ __forceinline__ void reduce_slot(TileCache& tc, int key, const SolidAt& q) {
    const int lane = threadIdx.x & 31;
    float val[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (key >= 0) {
        val[0] = -q.B * q.sx;
        val[1] = -q.B * q.sy;
        val[2] = -q.B * q.sz;
        val[3] = q.ay * val[2] - q.az * val[1];
        val[4] = q.az * val[0] - q.ax * val[2];
        val[5] = q.ax * val[1] - q.ay * val[0];
    }
    unsigned pending = __ballot_sync(FULL, key >= 0);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int kk = __shfl_sync(FULL, key, leader);
        const bool mine = key == kk;
        float v[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = mine ? val[c] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int c = 0; c < 6; ++c) v[c] += __shfl_xor_sync(FULL, v[c], off);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < 6; ++c) atomicAdd(&tc.acc[c][kk], (double)v[c]);
        pending &= ~__ballot_sync(FULL, mine);
    }
}

// ------------------------------------------------------------------------------------
// Asynchronous pull: each thread copies the 19 values it pulls for a plane straight into
// its own shared-memory slots (cp.async, 4-byte granules; 16-bit formats copy the aligned
// word holding the value). Only the issuing thread reads them back, so the pipeline
// needs no CTA barrier, and two planes of loads stay in flight per thread whatever the
// occupancy.
// ------------------------------------------------------------------------------------
constexpr int PSM_THREADS = TILE_X * TILE_Y;
constexpr int PSM_STAGES = 3;

__device__ __forceinline__ void cp_async4(uint32_t* dst, const void* src, bool pred) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    int n = pred ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Element index of the population pulled in direction I, and the wall flags of the link.
template <int I>
__device__ __forceinline__ long long pull_addr(const LbmArgs& a, const Nbr& nb, bool& wall, bool& wx,
                                               bool& wy, bool& wz) {
    constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
    wx = nb.wx[cx + 1];
    wy = nb.wy[cy + 1];
    wz = nb.wz[cz + 1];
    wall = wx || wy || wz;
    long long src = nb.xs[cx + 1] + (long long)a.nx * (nb.ys[cy + 1] + (long long)a.ny * nb.zs[cz + 1]);
    return wall ? (long long)OPP(I) * a.N + nb.cell : (long long)I * a.N + src;
}

// Per-plane pull plan of one node. Away from walls every source is node - off_i plus a
// periodic-wrap correction on the axes where the node sits on the first or last layer;
// next to a wall the general path (halfway bounce-back) is taken.
struct Plan {
    int cell;
    bool wall;                 // some link of this node crosses a wall
    int wxm, wxp, wym, wyp, wzm, wzp;  // wrap corrections for c = +1 (m) and c = -1 (p)
};

__device__ __forceinline__ void make_plan(const LbmArgs& a, int x, int y, int z, Plan& p) {
    const int nxy = a.nx * a.ny;
    p.cell = x + a.nx * y + nxy * z;
    bool w = false;
    p.wxm = p.wxp = p.wym = p.wyp = p.wzm = p.wzp = 0;
    if (x == 0) { if (a.per[0]) p.wxm = a.nx; else w = true; }
    if (x == a.nx - 1) { if (a.per[0]) p.wxp = -a.nx; else w = true; }
    if (y == 0) { if (a.per[1]) p.wym = nxy; else w = true; }
    if (y == a.ny - 1) { if (a.per[1]) p.wyp = -nxy; else w = true; }
    if (z == 0) { if (a.per[2]) p.wzm = (int)a.N; else w = true; }
    if (z == a.nz - 1) { if (a.per[2]) p.wzp = -(int)a.N; else w = true; }
    p.wall = w;
}

// element index of the population pulled in direction I (no wall on the link)
template <int I>
__device__ __forceinline__ int fast_elem(const LbmArgs& a, const Plan& p) {
    constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
    int src = p.cell - a.off[I];
    if (cx == 1) src += p.wxm;
    if (cx == -1) src += p.wxp;
    if (cy == 1) src += p.wym;
    if (cy == -1) src += p.wyp;
    if (cz == 1) src += p.wzm;
    if (cz == -1) src += p.wzp;
    return a.pN[I] + src;
}

template <class SS, int I>
struct IssueAll {
    static __device__ __forceinline__ void run(const LbmArgs& a, const typename SS::T* pin, const Plan& p,
                                               uint32_t* slot, bool pred) {
        int elem = 0;
        if (pred) {
            if (!p.wall) {
                elem = fast_elem<I>(a, p);
            } else {
                // general path (rare): halfway bounce-back where the link crosses a wall
                const int nxy = a.nx * a.ny;
                const int z = p.cell / nxy, y = (p.cell - z * nxy) / a.nx, x = p.cell - z * nxy - y * a.nx;
                Nbr nb;
                make_nbr(a, x, y, z, nb);
                bool wall, wx, wy, wz;
                elem = (int)pull_addr<I>(a, nb, wall, wx, wy, wz);
            }
        }
        uintptr_t q = reinterpret_cast<uintptr_t>(pin + elem);
        if (sizeof(typename SS::T) == 2) q &= ~(uintptr_t)3;
        cp_async4(slot + I * PSM_THREADS, reinterpret_cast<const void*>(q), pred);
        IssueAll<SS, I + 1>::run(a, pin, p, slot, pred);
    }
};
template <class SS>
struct IssueAll<SS, 19> {
    static __device__ __forceinline__ void run(const LbmArgs&, const typename SS::T*, const Plan&, uint32_t*,
                                               bool) {}
};

template <class SS>
__device__ __forceinline__ float decode(uint32_t w, int odd, float inv) {
    if (sizeof(typename SS::T) == 4) return __uint_as_float(w);
    unsigned short h = odd ? (unsigned short)(w >> 16) : (unsigned short)(w & 0xffffu);
    typename SS::T v;
    memcpy(&v, &h, 2);
    return SS::load(&v, inv);
}

template <class SS, int I>
struct ReadAll {
    static __device__ __forceinline__ void run(const LbmArgs& a, const Plan& p, const Nbr* nb,
                                               const uint32_t* slot, float* g) {
        const uint32_t w = slot[I * PSM_THREADS];
        if (!nb) {
            // parity of pN[I] + cell - off[I] (+ even wrap corrections for even sizes is
            // not assumed: use the exact element index)
            const int odd = sizeof(typename SS::T) == 2 ? (fast_elem<I>(a, p) & 1) : 0;
            g[I] = decode<SS>(w, odd, a.inv_scale);
        } else {
            bool wall, wx, wy, wz;
            long long addr = pull_addr<I>(a, *nb, wall, wx, wy, wz);
            float v = decode<SS>(w, (int)(addr & 1), a.inv_scale);
            if (wall) v += wall_term<I>(a.uw, wx, wy, wz);
            g[I] = v;
        }
        ReadAll<SS, I + 1>::run(a, p, nb, slot, g);
    }
};
template <class SS>
struct ReadAll<SS, 19> {
    static __device__ __forceinline__ void run(const LbmArgs&, const Plan&, const Nbr*, const uint32_t*,
                                               float*) {}
};

// ------------------------------------------------------------------------------------
// The fused PSM step: pull, moments, solid fractions, PSM collision (Eqs. psm1, lbePS,
// bk, btot), store, and the hydrodynamic force/torque of each solid (Eqs. forceSF,
// torqueSF) reduced warp -> tile (shared FP64) -> particle (global FP64 atomics).
// The collision is written around the non-equilibrium parts neq_i = g_i - geq_i:
//   f*_i = geq_i + (1 - (1-B_tot)/tau) neq_i + sum_k B_k Omega^s_{i,k},
//   Omega^s_{i,k} = neq_ibar - neq_i - (geq_i(rho,u) - geq_i(rho,u_k)).
// ------------------------------------------------------------------------------------
template <int STORE>
__global__ void __launch_bounds__(PSM_THREADS, 2) k_psm(const LbmArgs a) {
    using SS = Store<STORE>;
    using T = typename SS::T;
    const T* pin = (const T*)a.pop_in;
    T* pout = (T*)a.pop_out;
    extern __shared__ __align__(16) unsigned char psm_smem[];
    TileCache& tc = *reinterpret_cast<TileCache*>(psm_smem);
    uint32_t* stage = reinterpret_cast<uint32_t*>(psm_smem + ((sizeof(TileCache) + 15) & ~(size_t)15));
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * TILE_X, y0 = blockIdx.y * TILE_Y, z0 = blockIdx.z * TILE_Z;
    const int tile = (blockIdx.z * a.nty + blockIdx.y) * a.ntx + blockIdx.x;
    const int x = x0 + lane, y = y0 + warp;
    const bool valid_xy = x < a.nx && y < a.ny;

    // prologue: the first planes in flight while the tile's particles are cached
#pragma unroll
    for (int q = 0; q < PSM_STAGES - 1; ++q) {
        const int z = z0 + q;
        const bool pred = valid_xy && z < a.nz;
        Plan pl;
        if (pred) make_plan(a, x, y, z, pl);
        IssueAll<SS, 0>::run(a, pin, pl, stage + (q * 19) * PSM_THREADS + tid, pred);
        cp_async_commit();
    }
    const int cnt = min(a.tile_count[tile], a.tile_cap);
    load_tile(a, tc, tile, cnt, x0, y0, z0);
    __syncthreads();

    const float tau = a.tau, omega = a.omega;
    for (int iz = 0; iz < TILE_Z; ++iz) {
        {   // keep PSM_STAGES - 1 planes ahead in flight
            const int q = iz + PSM_STAGES - 1;
            const int z = z0 + q;
            const bool pred = q < TILE_Z && valid_xy && z < a.nz;
            Plan pl;
            if (pred) make_plan(a, x, y, z, pl);
            IssueAll<SS, 0>::run(a, pin, pl, stage + ((q % PSM_STAGES) * 19) * PSM_THREADS + tid, pred);
            cp_async_commit();
        }
        cp_async_wait<PSM_STAGES - 1>();
        const int z = z0 + iz;
        if (y >= a.ny || z >= a.nz) continue;  // uniform across the warp
        const bool valid = x < a.nx;
        const unsigned long long mask = cnt ? row_mask(a, tc, cnt, warp, iz) : 0ull;

        float g[19];
        Plan pl;
        pl.cell = 0;
        if (valid) {
            make_plan(a, x, y, z, pl);
            const uint32_t* slot = stage + ((iz % PSM_STAGES) * 19) * PSM_THREADS + tid;
            if (!pl.wall) {
                ReadAll<SS, 0>::run(a, pl, nullptr, slot, g);
            } else {
                Nbr nb;
                make_nbr(a, x, y, z, nb);
                ReadAll<SS, 0>::run(a, pl, &nb, slot, g);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 19; ++i) g[i] = 0.f;
        }
        Two t;
        t.ns = 0;
        t.total = 0;
        if (valid && mask) node_solids(a, tc, mask, lane, warp, iz, x, y, z, t);
        if (t.total > 2) atomicAdd(&a.status->solids_overflow, 1);

        // moments, Eqs. (rho), (momentum); rho = 1 + sum g (pairwise sums for ILP)
        const float drho = ((g[0] + (g[1] + g[2])) + ((g[3] + g[4]) + (g[5] + g[6]))) +
                           (((g[7] + g[8]) + (g[9] + g[10])) + ((g[11] + g[12]) + (g[13] + g[14]))) +
                           ((g[15] + g[16]) + (g[17] + g[18]));
        float jx = ((g[1] - g[2]) + (g[7] - g[8])) + ((g[9] - g[10]) + (g[11] - g[12])) + (g[13] - g[14]);
        float jy = ((g[3] - g[4]) + (g[7] - g[8])) + ((g[10] - g[9]) + (g[15] - g[16])) + (g[17] - g[18]);
        float jz = ((g[5] - g[6]) + (g[11] - g[12])) + ((g[14] - g[13]) + (g[15] - g[16])) + (g[18] - g[17]);
        const float rho = 1.0f + drho;
        if (a.has_force) {
            jx += 0.5f * a.F[0];
            jy += 0.5f * a.F[1];
            jz += 0.5f * a.F[2];
        }
        const float inv_rho = 1.0f / rho;
        const float ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
        const float usq = ux * ux + uy * uy + uz * uz;
        const float base = drho - rho * 1.5f * usq;

        // B_k, B_tot (Eqs. bk, btot)
        float B0 = 0.f, B1 = 0.f;
        if (t.ns > 0) B0 = t.b0 * (tau - 0.5f) / ((1.0f - t.b0) + (tau - 0.5f));
        if (t.ns > 1) B1 = t.b1 * (tau - 0.5f) / ((1.0f - t.b1) + (tau - 0.5f));
        const float Btot = fminf(B0 + B1, 1.0f);
        const float keep = 1.0f - (1.0f - Btot) * omega;
        const float force_w = (1.0f - Btot) * a.guo_pref;
        const float Fu = a.has_force ? a.F[0] * ux + a.F[1] * uy + a.F[2] * uz : 0.f;

        float neq[19], out[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float cu = (float)CX(i) * ux + (float)CY(i) * uy + (float)CZ(i) * uz;
            const float geq = TW(i) * (base + rho * (3.0f * cu + 4.5f * cu * cu));
            neq[i] = g[i] - geq;
            out[i] = geq + keep * neq[i];
            if (a.has_force) {
                const float cF = (float)CX(i) * a.F[0] + (float)CY(i) * a.F[1] + (float)CZ(i) * a.F[2];
                out[i] += force_w * TW(i) * (3.0f * (cF - Fu) + 9.0f * cu * cF);
            }
        }

        // solid operators, one solid at a time; the slot loop is warp-uniform
        for (int k = 0; k < 2; ++k) {
            const bool act = k < t.ns;
            if (!__any_sync(FULL, act)) break;
            SolidAt q;
            q.B = 0.f;
            q.ax = q.ay = q.az = 0.f;
            q.sx = q.sy = q.sz = 0.f;
            if (act) {
                solid_at(a, tc, k == 0 ? t.e0 : t.e1, k == 0 ? t.b0 : t.b1, lane, warp, iz, tau, q);
                const float dux = ux - q.ux, duy = uy - q.uy, duz = uz - q.uz;
                const float dusq = usq - q.usq;
#pragma unroll
                for (int i = 0; i < 19; ++i) {
                    const float cu = (float)CX(i) * ux + (float)CY(i) * uy + (float)CZ(i) * uz;
                    const float cuk = (float)CX(i) * q.ux + (float)CY(i) * q.uy + (float)CZ(i) * q.uz;
                    const float cdu = (float)CX(i) * dux + (float)CY(i) * duy + (float)CZ(i) * duz;
                    // geq_i(rho,u) - geq_i(rho,u_k)
                    const float dgeq = TW(i) * rho * (3.0f * cdu + 4.5f * (cu * cu - cuk * cuk) - 1.5f * dusq);
                    const float oms = neq[OPP(i)] - neq[i] - dgeq;
                    out[i] += q.B * oms;
                    if (CX(i)) q.sx += (float)CX(i) * oms;
                    if (CY(i)) q.sy += (float)CY(i) * oms;
                    if (CZ(i)) q.sz += (float)CZ(i) * oms;
                }
            }
            reduce_slot(tc, act ? (k == 0 ? t.e0 : t.e1) : -1, q);
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < 19; ++i) SS::store(pout + (a.pN[i] + pl.cell), out[i], a.scale);
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    for (int idx = tid; idx < 6 * cnt; idx += blockDim.x) {
        int e = idx / 6, c = idx % 6;
        double v = tc.acc[c][e];
        if (v != 0.0) {
            double* dst = c < 3 ? a.Fh + (long long)c * a.pcap : a.Mh + (long long)(c - 3) * a.pcap;
            atomicAdd(dst + tc.pid[e], v);
        }
    }
}

size_t psm_smem_bytes() {
    return ((sizeof(TileCache) + 15) & ~(size_t)15) + sizeof(uint32_t) * PSM_STAGES * 19 * PSM_THREADS;
}

// Solid fractions only (the same tile machinery), for inspection.
__global__ void __launch_bounds__(256) k_voxelize(const LbmArgs a, float* beta, int* ids, int* nsolid) {
    __shared__ TileCache tc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = blockIdx.x * TILE_X, y0 = blockIdx.y * TILE_Y, z0 = blockIdx.z * TILE_Z;
    const int tile = (blockIdx.z * a.nty + blockIdx.y) * a.ntx + blockIdx.x;
    const int cnt = min(a.tile_count[tile], a.tile_cap);
    load_tile(a, tc, tile, cnt, x0, y0, z0);
    __syncthreads();
    const int x = x0 + lane, y = y0 + warp;
    for (int iz = 0; iz < TILE_Z; ++iz) {
        const int z = z0 + iz;
        if (y >= a.ny || z >= a.nz) break;
        const unsigned long long mask = cnt ? row_mask(a, tc, cnt, warp, iz) : 0ull;
        if (x >= a.nx) continue;
        Two t;
        t.ns = 0;
        t.total = 0;
        if (mask) node_solids(a, tc, mask, lane, warp, iz, x, y, z, t);
        long long cell = x + (long long)a.nx * (y + (long long)a.ny * z);
        beta[2 * cell] = t.ns > 0 ? t.b0 : 0.f;
        beta[2 * cell + 1] = t.ns > 1 ? t.b1 : 0.f;
        ids[2 * cell] = t.ns > 0 ? tc.pid[t.e0] : -1;
        ids[2 * cell + 1] = t.ns > 1 ? tc.pid[t.e1] : -1;
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
    k_bin<<<(n + 127) / 128, 128, 0, s>>>(a, n, tile_count, tile_ids);
    return cudaGetLastError();
}

template <int STORE>
static cudaError_t launch_psm_t(const LbmArgs& a, cudaStream_t s) {
    static bool configured = false;
    const size_t smem = psm_smem_bytes();
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_psm<STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_psm<STORE><<<tile_grid(a), PSM_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_psm(const LbmArgs& a, int store, cudaStream_t s) {
    if (store == LEDDS_STORE_F32) return launch_psm_t<LEDDS_STORE_F32>(a, s);
    if (store == LEDDS_STORE_F16) return launch_psm_t<LEDDS_STORE_F16>(a, s);
    return launch_psm_t<LEDDS_STORE_BF16>(a, s);
}

cudaError_t launch_voxelize(const LbmArgs& a, float* beta, int* ids, int* nsolid, cudaStream_t s) {
    k_voxelize<<<tile_grid(a), 256, 0, s>>>(a, beta, ids, nsolid);
    return cudaGetLastError();
}

}  // namespace ledds
