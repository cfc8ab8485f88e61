// psm.cuh -- the fused PSM kernel of one lattice tile (Secs. 2.3-2.4, Table 1
// "Compute solid fractions", "LBM-PSM collision and streaming", "Force reduction"),
// shared by the translation units that instantiate it: lbm.cu (two-lattice pull),
// psm_aa.cu (the in-place AA pattern) and psm_wide.cu (64-bit population offsets).
#pragma once

#include <type_traits>
#include <utility>

#include "internal.cuh"

namespace ledds {

cudaError_t launch_psm_aa(const LbmArgs& a, const PsmMaps* m, int store, cudaStream_t s);    // psm_aa.cu
cudaError_t launch_psm_wide(const LbmArgs& a, const PsmMaps* m, int store, cudaStream_t s);  // psm_wide.cu

constexpr unsigned FULL = 0xffffffffu;

// Explicitly rounded FP32 operations: the collision is written with these so that every
// instantiation of the kernel (pull route, step form, offset width) rounds identically
// (no contraction or reassociation left to the compiler).
__device__ __forceinline__ float fm(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float mu(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ad(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sb(float a, float b) { return __fsub_rn(a, b); }
// Square root by the hardware approximation (relative error about 2^-23, exact at 0): the
// distance solid fraction (R + R_c - d) / (2 R_c) needs no correctly rounded root.
__device__ __forceinline__ float sqrt_apx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
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

__device__ __forceinline__ float reach_of(const LbmArgs& a, int shape, double R, double Rb) {
    // distance method: beta > 0 iff |x - r| < R + R_c; subdivision: samples lie within
    // 0.78 of the node, use the bounding radius plus the cell half-diagonal.
    if (shape == LEDDS_SPHERE && a.voxel == LEDDS_VOXEL_DISTANCE) return (float)R + a.Rc + 1e-3f;
    return (float)Rb + 0.8661f + 1e-3f;
}

// ------------------------------------------------------------------------------------
// Per-tile particle cache and solid fractions (Sec. 2.4)
// ------------------------------------------------------------------------------------
// Per-tile particle cache. The hot fields are packed in float4 records so one 128-bit
// shared load (a broadcast: every lane reads the same entry) fetches a whole record.
struct TileCache {
    float4 pos[MAX_TILE_CAP];     // centre minus tile origin (FP32, minimum image), radius
    float4 vel[MAX_TILE_CAP];     // velocity, squared reach of the solid fraction
    float4 spin[MAX_TILE_CAP];    // angular velocity, particle id (bits)
    int shape[MAX_TILE_CAP];
    float R2[MAX_TILE_CAP];       // fl32(R*R) of the subdivision predicate
    double p[3][MAX_TILE_CAP];    // centre (FP64) for the exact subdivision path
    float m[9][MAX_TILE_CAP];     // ellipsoid rows fl32(d_j / semi_j)
    float acc[6][MAX_TILE_CAP];   // force and torque sums of this tile (FP32: native shared atomics)
    float so[16];                 // subdivision sample offsets (2m + 1 - n)/(2n)
    float ims[MAX_TILE_CAP];      // ellipsoid: 1 / smallest semi-axis (norm of the m rows)
    float G[MAX_TILE_CAP];        // ellipsoid: largest |M c|^2 over the subdivision sample box
    float4 sdw[MAX_TILE_CAP];     // ellipsoid: y-z shadow f11, 2 f12, f22 and its grown bound
    float spx[TILE_Y][32];        // subdivision counts: x offsets of a warp's nodes
    int scnt[TILE_Y][32];         // subdivision counts: samples decided by the predicate
};

__device__ __forceinline__ int tc_pid(const TileCache& tc, int e) { return __float_as_int(tc.spin[e].w); }

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

static __device__ void load_tile(const LbmArgs& a, TileCache& tc, int tile, int cnt, int x0, int y0,
                          int z0) {
    if (threadIdx.x < 16) {
        const int n = a.subdiv_n;
        tc.so[threadIdx.x] = (int)threadIdx.x < n ? __fdiv_rn((float)(2 * (int)threadIdx.x + 1 - n), (float)(2 * n)) : 0.0f;
    }
    const double org[3] = {(double)x0, (double)y0, (double)z0};
    const double Ls[3] = {(double)a.nx, (double)a.ny, (double)a.nz};
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int k = a.tile_ids[(long long)tile * a.tile_cap + e];
        int sh = a.shape[k];
        tc.shape[e] = sh;
        float r[3], v[3], w[3];
        for (int c = 0; c < 3; ++c) {
            double pc = a.st[(SP + c) * a.pcap + k];
            tc.p[c][e] = pc;
            r[c] = (float)min_image_d(pc - org[c], a.per[c], Ls[c]);
            v[c] = (float)a.st[(SV + c) * a.pcap + k];
            w[c] = (float)a.st[(SW + c) * a.pcap + k];
        }
        double R = sh == LEDDS_SPHERE ? a.radius[k] : a.bound[k];
        tc.R2[e] = __double2float_rn(R * R);
        float reach = reach_of(a, sh, a.radius[k], a.bound[k]);
        tc.pos[e] = make_float4(r[0], r[1], r[2], (float)R);
        tc.vel[e] = make_float4(v[0], v[1], v[2], reach * reach);
        tc.spin[e] = make_float4(w[0], w[1], w[2], __int_as_float(k));
        if (sh == LEDDS_ELLIPSOID) {
            for (int j = 0; j < 3; ++j)
                for (int c = 0; c < 3; ++c)
                    tc.m[3 * j + c][e] = __double2float_rn(
                        a.st[(ST + 3 * j + c) * a.pcap + k] / a.semi[j * a.pcap + k]);
            const double smin = fmin(a.semi[k], fmin(a.semi[a.pcap + k], a.semi[2 * a.pcap + k]));
            tc.ims[e] = (float)(1.0 / smin);
            // corners c = h (1, s1, s2), s_k = +-1, of the sample box (c and -c alike)
            const double h = (double)(a.subdiv_n - 1) / (double)(2 * a.subdiv_n);
            double g = 0.0;
            for (int sg = 0; sg < 4; ++sg) {
                const double s1 = (sg & 1) ? -1.0 : 1.0, s2 = (sg & 2) ? -1.0 : 1.0;
                double v = 0.0;
                for (int j = 0; j < 3; ++j) {
                    const double r = (double)tc.m[3 * j][e] + s1 * (double)tc.m[3 * j + 1][e] +
                                     s2 * (double)tc.m[3 * j + 2][e];
                    v += r * r;
                }
                g = fmax(g, v);
            }
            tc.G[e] = (float)(g * h * h * 1.0001);
            // Shadow on the y-z plane: the smallest |M (X, dy, dz)|^2 over X is the Schur
            // complement quadratic f11 dy^2 + 2 f12 dy dz + f22 dz^2 of M^T M. A node's
            // samples lie within h sqrt(2) of the row (ly, lz) in y-z, and the square root
            // of the quadratic grows by at most 1/smallest semi-axis per unit distance, so a
            // row whose value is at least (1 + h sqrt(2) / s_min)^2 (with margins) has no
            // sample inside at any of its nodes.
            double Q[3][3];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    double v = 0.0;
                    for (int j = 0; j < 3; ++j) v += (double)tc.m[3 * j + r][e] * (double)tc.m[3 * j + c][e];
                    Q[r][c] = v;
                }
            const double f11 = Q[1][1] - Q[0][1] * Q[0][1] / Q[0][0];
            const double f12 = Q[1][2] - Q[0][1] * Q[0][2] / Q[0][0];
            const double f22 = Q[2][2] - Q[0][2] * Q[0][2] / Q[0][0];
            const double grow = 1.0 + (h * 1.41421356237 + 1e-3) / smin + 1e-3;
            tc.sdw[e] = make_float4((float)f11, (float)(2.0 * f12), (float)f22, (float)(grow * grow * 1.001));
        } else {
            tc.sdw[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int c = 0; c < 6; ++c) tc.acc[c][e] = 0.0f;
    }
}

// Subdivision predicate (Sec. 2.4): a sample at offset (dx, dy, dz) from the centre is
// strictly inside the solid. Evaluated in FP32 with explicit round-to-nearest intrinsics
// in a fixed order (no contraction), so each decision is reproducible.
constexpr float SUBDIV_MARGIN = 1e-3f;

__device__ __forceinline__ bool subdiv_pred_sphere(float dx, float yy, float zz, float R2) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), yy), zz) < R2;
}
__device__ __forceinline__ bool subdiv_pred_ell(const float (&mm)[9], float dx, float dy, float dz) {
    const float t0 = __fadd_rn(__fmul_rn(mm[0], dx), __fmul_rn(mm[1], dy));
    const float t1 = __fadd_rn(__fmul_rn(mm[3], dx), __fmul_rn(mm[4], dy));
    const float t2 = __fadd_rn(__fmul_rn(mm[6], dx), __fmul_rn(mm[7], dy));
    const float q0 = __fadd_rn(t0, __fmul_rn(mm[2], dz));
    const float q1 = __fadd_rn(t1, __fmul_rn(mm[5], dz));
    const float q2 = __fadd_rn(t2, __fmul_rn(mm[8], dz));
    return __fadd_rn(__fadd_rn(__fmul_rn(q0, q0), __fmul_rn(q1, q1)), __fmul_rn(q2, q2)) < 1.0f;
}

// Solid fraction of cached particle e at a node, (dx,dy,dz) = node - centre (FP32), where
// it follows from the distance (Eq. naiveSolidFrac) or from the exact early-outs of the
// subdivision method; *exact is set when the subdivision count itself is needed.
__device__ __forceinline__ float beta_quick(const LbmArgs& a, const TileCache& tc, int e, float dx, float dy,
                                            float dz, float R, bool* exact) {
    const int sh = tc.shape[e];
    const float d2 = fm(dz, dz, fm(dy, dy, mu(dx, dx)));
    *exact = false;
    if (sh == LEDDS_SPHERE && a.voxel == LEDDS_VOXEL_DISTANCE) {
        // Eq. (naiveSolidFrac): (R + R_c - d) / (2 R_c), clamped
        const float dsc = sb(ad(R, a.Rc), sqrt_apx(d2));
        return fminf(fmaxf(mu(dsc, a.inv2Rc), 0.0f), 1.0f);
    }
    const int n = a.subdiv_n;
    const float h = (float)(n - 1) / (float)(2 * n);  // largest sample offset
    const float hd = 1.7320508f * h;                  // sample-to-node distance bound
    // exact early-outs (margins far above FP32 rounding): no sample can be inside ...
    const float far = R + hd + 1e-3f;
    if (d2 > far * far) return 0.0f;
    if (sh == LEDDS_SPHERE) {
        const float nearr = R - hd - 1e-3f;
        if (nearr > 0.0f && d2 < nearr * nearr) return 1.0f;  // ... or every sample is
    } else {
        // q = M p (M rows d_j / semi_j), w = M^T q. Over the box of samples p + c, |c_k| <= h,
        // |M (p + c)|^2 = |q|^2 + 2 w.c + |M c|^2 lies between |q|^2 - 2 h |w|_1 and
        // |q|^2 + 2 h |w|_1 + G, G = max over the box of |M c|^2 (its largest corner, per
        // particle): beyond 1 by the margin no sample is inside, below it every one is (the
        // margins are far above the FP32 rounding of either side)
        const float q0 = tc.m[0][e] * dx + tc.m[1][e] * dy + tc.m[2][e] * dz;
        const float q1 = tc.m[3][e] * dx + tc.m[4][e] * dy + tc.m[5][e] * dz;
        const float q2 = tc.m[6][e] * dx + tc.m[7][e] * dy + tc.m[8][e] * dz;
        const float s2 = q0 * q0 + q1 * q1 + q2 * q2;
        const float w0 = tc.m[0][e] * q0 + tc.m[3][e] * q1 + tc.m[6][e] * q2;
        const float w1 = tc.m[1][e] * q0 + tc.m[4][e] * q1 + tc.m[7][e] * q2;
        const float w2 = tc.m[2][e] * q0 + tc.m[5][e] * q1 + tc.m[8][e] * q2;
        const float l1 = 2.0f * h * (fabsf(w0) + fabsf(w1) + fabsf(w2));
        const float slack = 1e-3f + 1e-5f * (s2 + l1);
        if (s2 - l1 > 1.0f + slack) return 0.0f;
        if (s2 + l1 + tc.G[e] < 1.0f - slack) return 1.0f;
    }
    *exact = true;
    return 0.0f;
}

// Row prefilter: which cached particles can touch the x-row (ly, lz) of this tile.
// MI: a node-particle offset may need a periodic wrap (a.mi); false when no axis does
// (known at compile time).
template <bool MI>
__device__ __forceinline__ float mimg(float d, int per, float L) {
    if constexpr (MI) return min_image_f(d, per, L);
    else return d;
}

template <bool MI>
__device__ __forceinline__ unsigned long long row_mask(const LbmArgs& a, const TileCache& tc,
                                                       int cnt, int ly, int lz) {
    const int lane = threadIdx.x & 31;
    unsigned long long mask = 0ull;
    for (int base = 0; base < cnt; base += 32) {
        int e = base + lane;
        bool hit = false;
        if (e < cnt) {
            const float4 ps = tc.pos[e];
            float dy = mimg<MI>((float)ly - ps.y, a.mi[1], (float)a.ny);
            float dz = mimg<MI>((float)lz - ps.z, a.mi[2], (float)a.nz);
            hit = dy * dy + dz * dz < tc.vel[e].w;
            if constexpr (MI) {
                // an ellipsoid: its shadow on the y-z plane, grown to cover the samples of
                // the row's nodes (sdw.w 0: not an ellipsoid)
                const float4 sd = tc.sdw[e];
                hit = hit && (sd.w == 0.0f || fm(sd.x * dy, dy, fm(sd.y * dy, dz, mu(sd.z * dz, dz))) < sd.w);
            }
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
    if (b != bw) return b > bw;
    return tc_pid(tc, e) < tc_pid(tc, ew);  // a tie: the lower particle id first
}

// floor and ceiling of |v| < 2^22 as integers, by one directed-rounding addition
__device__ __forceinline__ int floor_small(float v) {
    return __float_as_int(__fadd_rd(v, 12582912.0f)) - 0x4B400000;
}
__device__ __forceinline__ int ceil_small(float v) {
    return __float_as_int(__fadd_ru(v, 12582912.0f)) - 0x4B400000;
}

// One sample row (fixed y and z offsets dy, dz) of the subdivision count. Along it the
// squared normalised radius is the quadratic F(X) = A X^2 + 2 B X + C of the x offset X,
// smallest (Fmin) at xc = -B/A (spheres: X^2 + dy^2 + dz^2 against R^2). The row keeps the
// interval around xc where F < 1 - 1e-3, shrunk by 2e-4, and the one where F <= 1 + 1e-3,
// grown by 2e-4, as fractional sample indices of a node at x offset 0 (sample i of a node
// at offset qx sits at X = qx + (i - (n - 1)/2)/n).
struct SubRow {
    float ilo, ihi, olo, ohi;  // inner and outer interval (empty: lo > hi)
    float dy, dz, yy, zz;
};

__device__ __forceinline__ void subdiv_row(const TileCache& tc, bool sph, const float (&mm)[9], float iA,
                                           float lo, float hi, float py, float pz, int j, int q, float fn,
                                           float t0, SubRow& r) {
    r.dy = __fadd_rn(py, tc.so[j]);
    r.dz = __fadd_rn(pz, tc.so[q]);
    r.yy = __fmul_rn(r.dy, r.dy);
    r.zz = __fmul_rn(r.dz, r.dz);
    float xc = 0.0f, Fmin;
    if (sph) {
        Fmin = r.yy + r.zz;
    } else {
        const float w0 = mm[1] * r.dy + mm[2] * r.dz, w1 = mm[4] * r.dy + mm[5] * r.dz,
                    w2 = mm[7] * r.dy + mm[8] * r.dz;
        const float B = mm[0] * w0 + mm[3] * w1 + mm[6] * w2;
        const float C = w0 * w0 + w1 * w1 + w2 * w2;
        xc = -B * iA;
        Fmin = C + B * xc;
    }
    r.olo = r.ilo = 1e4f;
    r.ohi = r.ihi = -1e4f;
    if (Fmin <= hi) {
        // square roots to about 1e-7 relative (the slack is 1e-5 relative plus 2e-4)
        const float vo = fmaxf((hi - Fmin) * iA, 1e-30f), vi = fmaxf((lo - Fmin) * iA, 1e-30f);
        const float ro = vo * rsqrtf(vo) * (1.0f + 1e-5f) + 2e-4f;
        const float c = xc * fn + t0;
        r.olo = c - ro * fn;
        r.ohi = c + ro * fn;
        if (Fmin < lo) {
            const float ri = vi * rsqrtf(vi) * (1.0f - 1e-5f) - 2e-4f;
            if (ri > 0.0f) {
                r.ilo = c - ri * fn;
                r.ihi = c + ri * fn;
            }
        }
    }
}

// Samples of row r inside the solid for the node at x offset qx (qxn = qx n): those in the
// inner interval by index arithmetic, the FP32 predicate for those between the intervals.
__device__ __forceinline__ int subdiv_row_count(const TileCache& tc, const SubRow& r, bool sph,
                                                const float (&mm)[9], float thr, float qx, float qxn,
                                                int n) {
    const int oA = max(0, ceil_small(r.olo - qxn)), oB = min(n - 1, floor_small(r.ohi - qxn));
    const int iA = max(0, ceil_small(r.ilo - qxn)), iB = min(n - 1, floor_small(r.ihi - qxn));
    int c = 0, e1 = oB + 1, s2 = oB + 1;  // predicate on [oA, e1) and [s2, oB]
    if (iA <= iB) {
        c = iB - iA + 1;
        e1 = iA;
        s2 = iB + 1;
    }
    for (int i = oA; i < e1; ++i) {
        const float dx = __fadd_rn(qx, tc.so[i]);
        c += sph ? subdiv_pred_sphere(dx, r.yy, r.zz, thr) : subdiv_pred_ell(mm, dx, r.dy, r.dz);
    }
    for (int i = s2; i <= oB; ++i) {
        const float dx = __fadd_rn(qx, tc.so[i]);
        c += sph ? subdiv_pred_sphere(dx, r.yy, r.zz, thr) : subdiv_pred_ell(mm, dx, r.dy, r.dz);
    }
    return c;
}

// Exact subdivision counts (Sec. 2.4) for the lanes in `need`: n^3 samples at offsets
// (2m+1-n)/(2n) around each node, a sample counting when the FP32 predicate puts it
// inside. The nodes of a warp lie on one x-row, so their y and z offsets from the centre
// (FP64 minimum image, rounded to FP32) are the same and so are the n^2 sample rows: the
// margins of a row's intervals (SubRow) are far above the rounding of the set-up and of
// the predicate (about 1e-5), so a sample in the inner interval is inside by the
// predicate, one outside the outer is not, and only samples between the two run it. The
// rows are taken 32 at a time, one per lane. The samples of the needing nodes Lmin..Lmax
// lie on one grid along x (node L's sample i is the (L - Lmin) n + i-th), so a lane maps
// its row's intervals onto that grid once, runs the predicate on the few samples between
// them (adding hits to the node's shared counter), and the warp sums each needing node's
// overlap with the inner interval. Where the nodes' offsets do not lie on one grid (they
// would take different periodic images: tiny periodic boxes) each node is counted alone.
__device__ __forceinline__ float subdiv_lanes(const LbmArgs& a, TileCache& tc, int e, unsigned need,
                                              bool exact, int x, int y, int z, float b) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = a.subdiv_n, nn = n * n;
    // offsets node - centre: the needing lanes take their own x, two other lanes (when
    // there are two) the row's y and z, so the FP64 work is done once
    float px, py, pz;
    const unsigned spare = ~need;
    if (__popc(spare) >= 2) {
        const int ly = __ffs(spare) - 1;
        const int lz = __ffs(spare & (spare - 1)) - 1;
        const int ax = lane == ly ? 1 : (lane == lz ? 2 : 0);
        const int cc = ax == 0 ? x : (ax == 1 ? y : z);
        const double L = ax == 0 ? (double)a.nx : (ax == 1 ? (double)a.ny : (double)a.nz);
        const float v = __double2float_rn(min_image_d((double)cc - tc.p[ax][e], a.per[ax], L));
        px = v;
        py = __shfl_sync(0xffffffffu, v, ly);
        pz = __shfl_sync(0xffffffffu, v, lz);
    } else {
        px = __double2float_rn(min_image_d((double)x - tc.p[0][e], a.per[0], (double)a.nx));
        py = __double2float_rn(min_image_d((double)y - tc.p[1][e], a.per[1], (double)a.ny));
        pz = __double2float_rn(min_image_d((double)z - tc.p[2][e], a.per[2], (double)a.nz));
    }
    const bool sph = tc.shape[e] == LEDDS_SPHERE;
    float mm[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) mm[k] = sph ? 0.0f : tc.m[k][e];
    const float iA = sph ? 1.0f : __frcp_rn(mm[0] * mm[0] + mm[3] * mm[3] + mm[6] * mm[6]);
    const float thr = sph ? tc.R2[e] : 1.0f;
    const float lo = thr * (1.0f - SUBDIV_MARGIN), hi = thr * (1.0f + SUBDIV_MARGIN);
    const float fn = (float)n, t0 = 0.5f * (float)(n - 1);
    const unsigned mgc = 0xffffffffu / (unsigned)n + 1u;  // v / n = umulhi(v, mgc) for v < 2^16
    const bool mine = (need >> lane) & 1u;
    const int Lmin = __ffs(need) - 1, Lmax = 31 - __clz(need);
    const float p0 = __shfl_sync(0xffffffffu, px, Lmin);  // x offset of node Lmin
    const bool grid = __all_sync(0xffffffffu, !mine || fabsf(px - p0 - (float)(lane - Lmin)) < 1e-3f);
    const float bn = p0 * fn;                  // node Lmin's first sample at grid index 0
    const int S = (Lmax - Lmin + 1) * n;       // grid samples
    int count = 0;
    if (grid) {
        tc.spx[warp][lane] = px;
        tc.scnt[warp][lane] = 0;
        __syncwarp();
    }
    for (int r0 = 0; r0 < nn; r0 += 32) {
        const int jq = r0 + lane;
        SubRow rw;
        rw.olo = rw.ilo = 1e4f;
        rw.ohi = rw.ihi = -1e4f;
        rw.dy = rw.dz = rw.yy = rw.zz = 0.0f;
        if (jq < nn) {
            const int j = (int)__umulhi((unsigned)jq, mgc), q = jq - j * n;
            subdiv_row(tc, sph, mm, iA, lo, hi, py, pz, j, q, fn, t0, rw);
        }
        if (grid) {
            const int oA = max(0, ceil_small(rw.olo - bn)), oB = min(S - 1, floor_small(rw.ohi - bn));
            int gA = max(0, ceil_small(rw.ilo - bn)), gB = min(S - 1, floor_small(rw.ihi - bn));
            int e1 = oB + 1, s2 = oB + 1;  // predicate on [oA, e1) and [s2, oB]
            if (gA <= gB) {
                e1 = gA;
                s2 = gB + 1;
            } else {
                gA = 0;
                gB = -1;
            }
            for (int g = oA; g <= oB; ++g) {
                if (g == e1) g = s2;
                if (g > oB) break;
                const int k = (int)__umulhi((unsigned)g, mgc), L = Lmin + k;
                if ((need >> L) & 1u) {
                    const float dx = __fadd_rn(tc.spx[warp][L], tc.so[g - k * n]);
                    if (sph ? subdiv_pred_sphere(dx, rw.yy, rw.zz, thr) : subdiv_pred_ell(mm, dx, rw.dy, rw.dz))
                        atomicAdd(&tc.scnt[warp][L], 1);
                }
            }
            unsigned todo = need;
            while (todo) {
                const int L = __ffs(todo) - 1;
                todo &= todo - 1u;
                const int w0 = (L - Lmin) * n;
                const int ov = max(0, min(gB, w0 + n - 1) - max(gA, w0) + 1);
                const int sum = __reduce_add_sync(0xffffffffu, ov);
                if (lane == L) count += sum;
            }
        } else {
            unsigned todo = need;
            while (todo) {
                const int l = __ffs(todo) - 1;
                todo &= todo - 1u;
                const float qx = __shfl_sync(0xffffffffu, px, l);
                const int c = jq < nn ? subdiv_row_count(tc, rw, sph, mm, thr, qx, qx * fn, n) : 0;
                const int sum = __reduce_add_sync(0xffffffffu, c);
                if (lane == l) count += sum;
            }
        }
    }
    if (grid) {
        __syncwarp();
        count += tc.scnt[warp][lane];
        __syncwarp();  // the counters are reused by this warp's next call
    }
    return exact ? (float)count / (float)(n * n * n) : b;
}

// Called by the whole warp (the row mask is uniform); lanes with valid false take no part
// beyond the warp-wide subdivision counts.
// SPHD: every particle is a sphere with distance-based solid fractions and no offset
// needs a periodic wrap (known at compile time: the subdivision, ellipsoid and wrap code
// is left out).
template <bool SPHD>
__device__ __forceinline__ void node_solids(const LbmArgs& a, TileCache& tc,
                                            unsigned long long mask, int lx, int ly, int lz, int x,
                                            int y, int z, bool valid, Two& t) {
    t.ns = 0;
    t.total = 0;
    t.e0 = t.e1 = 0;
    t.b0 = t.b1 = 0.f;
    while (mask) {
        const int e = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        const float4 ps = tc.pos[e];
        float dx = mimg<!SPHD>((float)lx - ps.x, a.mi[0], (float)a.nx);
        float dy = mimg<!SPHD>((float)ly - ps.y, a.mi[1], (float)a.ny);
        float dz = mimg<!SPHD>((float)lz - ps.z, a.mi[2], (float)a.nz);
        float b;
        if constexpr (SPHD) {
            // Eq. (naiveSolidFrac), as in beta_quick
            const float d2 = fm(dz, dz, fm(dy, dy, mu(dx, dx)));
            const float dsc = sb(ad(ps.w, a.Rc), sqrt_apx(d2));
            b = valid ? fminf(fmaxf(mu(dsc, a.inv2Rc), 0.0f), 1.0f) : 0.0f;
        } else {
            bool exact = false;
            b = valid ? beta_quick(a, tc, e, dx, dy, dz, ps.w, &exact) : 0.0f;
            if (a.subdiv_any) {  // uniform: distance-fraction spheres never need counts
                const unsigned need = __ballot_sync(0xffffffffu, exact);
                if (need) b = subdiv_lanes(a, tc, e, need, exact, x, y, z, b);  // uniform branch
            }
        }
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

// One solid's data at a node: B_k (Eq. bk), surface velocity u_k = v_k + w_k x (x - r_k)
// and the arm x - r_k.
struct SolidAt {
    float B, ux, uy, uz, ax, ay, az;
};

template <bool MI>
__device__ __forceinline__ void solid_at(const LbmArgs& a, const TileCache& tc, int e, float b, int lx,
                                         int ly, int lz, SolidAt& q) {
    const float4 ps = tc.pos[e], vs = tc.vel[e], ws = tc.spin[e];
    q.ax = mimg<MI>(sb((float)lx, ps.x), a.mi[0], (float)a.nx);
    q.ay = mimg<MI>(sb((float)ly, ps.y), a.mi[1], (float)a.ny);
    q.az = mimg<MI>(sb((float)lz, ps.z), a.mi[2], (float)a.nz);
    const float th = sb(a.tau, 0.5f);
    q.B = __fdividef(mu(b, th), ad(sb(1.0f, b), th));
    q.ux = ad(vs.x, sb(mu(ws.y, q.az), mu(ws.z, q.ay)));
    q.uy = ad(vs.y, sb(mu(ws.z, q.ax), mu(ws.x, q.az)));
    q.uz = ad(vs.z, sb(mu(ws.x, q.ay), mu(ws.y, q.ax)));
}

// Force and torque of one node-solid pair, Eqs. (forceSF), (torqueSF):
// F = -B sum_i Omega^s_i c_i, M = arm x F. The direction sum has the closed form
// sum_i Omega^s_i c_i = F_fluid - rho (u - u_k) (momentum exchange: sum_i neq_i c_i =
// -F_fluid/2 and sum_i (geq_i(rho,u) - geq_i(rho,u_k)) c_i = rho (u - u_k)), so
// F = B (rho (u - u_k) - F_fluid).
__device__ __forceinline__ void solid_force(const SolidAt& q, float rho, float dux, float duy, float duz,
                                            const LbmArgs& a, float v[6]) {
    const float fx = a.has_force ? a.F[0] : 0.f, fy = a.has_force ? a.F[1] : 0.f;
    const float fz = a.has_force ? a.F[2] : 0.f;
    v[0] = mu(q.B, sb(mu(rho, dux), fx));
    v[1] = mu(q.B, sb(mu(rho, duy), fy));
    v[2] = mu(q.B, sb(mu(rho, duz), fz));
    v[3] = sb(mu(q.ay, v[2]), mu(q.az, v[1]));
    v[4] = sb(mu(q.az, v[0]), mu(q.ax, v[2]));
    v[5] = sb(mu(q.ax, v[1]), mu(q.ay, v[0]));
}

// Warp-aggregated addition of per-lane (key, 6 values) into the tile accumulators: one
// butterfly per distinct key present in the warp (lanes with key < 0 take no part).
// Inlined in the sphere kernel (no call frame), out of line in the general kernel (whose
// register budget it would otherwise strain): warp_flush<true> / warp_flush<false>.
__device__ __forceinline__ void warp_flush_body(TileCache& tc, int key, const float val[6]) {
    const int lane = threadIdx.x & 31;
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
            for (int c = 0; c < 6; ++c) atomicAdd(&tc.acc[c][kk], v[c]);
        pending &= ~__ballot_sync(FULL, mine);
    }
}
static __device__ __noinline__ void warp_flush_call(TileCache& tc, int key, const float val[6]) {
    warp_flush_body(tc, key, val);
}
template <bool INL>
__device__ __forceinline__ void warp_flush(TileCache& tc, int key, const float val[6]) {
    if constexpr (INL) warp_flush_body(tc, key, val);
    else warp_flush_call(tc, key, val);
}


// ------------------------------------------------------------------------------------
// Pulling the populations of a node. Two routes with one result:
//  - staged: per z-plane of a tile, the tensor engine (TMA) copies one box per direction
//    (the tile's 8 rows shifted by -c_i) from the population array into a ring of
//    shared-memory stages, each guarded by a pair of mbarriers (data landed / stage read
//    by every warp); each warp reads its own row back at fixed offsets;
//  - direct: per-thread loads from global memory, for lattices whose rows are not a
//    multiple of 16 bytes, batch members, the rows on a lattice face and the lanes at
//    the x ends of the lattice (periodic wraps and halfway bounce-back).
// ------------------------------------------------------------------------------------
constexpr int PSM_THREADS = TILE_X * TILE_Y;

// Calls f(std::integral_constant<int, I>) for I = 0 .. N-1 (a compile-time loop over the
// directions, so every table entry folds into an immediate).
template <class F, int... Is>
__device__ __forceinline__ void static_for_seq(F&& f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_seq(f, std::make_integer_sequence<int, N>{});
}


// Per-plane pull plan of one node: the source of direction I is node - off_I, plus a
// periodic-wrap correction on an axis where the node sits on the first or last layer; a
// link that leaves the lattice through a wall (bit of bw: x low/high 1/2, y 4/8, z 16/32)
// pulls the node's own opposite population instead (halfway bounce-back).
struct Plan {
    int cell;
    unsigned bw;                       // wall faces next to this node
    int wxm, wxp, wym, wyp, wzm, wzp;  // wrap corrections for c = +1 (m) and c = -1 (p)
};

__device__ __forceinline__ void make_plan(const LbmArgs& a, int x, int y, int z, Plan& p) {
    const int nxy = a.nx * a.ny;
    p.cell = x + a.nx * y + nxy * z;
    unsigned b = 0;
    p.wxm = p.wxp = p.wym = p.wyp = p.wzm = p.wzp = 0;
    if (x == 0) { if (a.per[0]) p.wxm = a.nx; else b |= 1u; }
    if (x == a.nx - 1) { if (a.per[0]) p.wxp = -a.nx; else b |= 2u; }
    if (y == 0) { if (a.per[1]) p.wym = nxy; else b |= 4u; }
    if (y == a.ny - 1) { if (a.per[1]) p.wyp = -nxy; else b |= 8u; }
    if (z == 0) { if (a.per[2]) p.wzm = (int)a.N; else b |= 16u; }
    if (z == a.nz - 1) { if (a.per[2]) p.wzp = -(int)a.N; else b |= 32u; }
    p.bw = b;
}

// The plan of a node known to be off every lattice face (no wrap, no wall link).
__device__ __forceinline__ void cell_plan(const LbmArgs& a, int x, int y, int z, Plan& p) {
    p.cell = x + a.nx * (y + a.ny * z);
    p.bw = 0u;
    p.wxm = p.wxp = p.wym = p.wyp = p.wzm = p.wzp = 0;
}

// Walls crossed by the link of direction I (the axis flags of wall_term).
template <int I>
__device__ __forceinline__ void link_walls(const Plan& p, bool& wx, bool& wy, bool& wz) {
    constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
    wx = (cx == 1 && (p.bw & 1u)) || (cx == -1 && (p.bw & 2u));
    wy = (cy == 1 && (p.bw & 4u)) || (cy == -1 && (p.bw & 8u));
    wz = (cz == 1 && (p.bw & 16u)) || (cz == -1 && (p.bw & 32u));
}

// Element offsets into the population array: 32-bit, or 64-bit under PSM_W64; the offset
// of plane i is then i N computed in 64 bits instead of the 32-bit table entry.
template <int MODE>
using PsmIdx = std::conditional_t<psm_w64(MODE), long long, int>;
template <int MODE>
__device__ __forceinline__ PsmIdx<MODE> plane_at(const LbmArgs& a, int i) {
    if constexpr (psm_w64(MODE)) return (long long)i * a.N;
    else return a.pN[i];
}

// Element index of the population f_I(x) a step of form MODE reads; WALLS: some link of
// the warp may cross a wall (uniform choice of the caller).
//   PSM_AB:      f*_I(x - c_I) in plane I, or at a wall f*_opp(I)(x) (halfway bounce-back);
//   PSM_AA_EVEN: f_I(x) itself, in plane I at x (no streaming in this step);
//   PSM_AA_ODD:  f*_I(x - c_I), kept by the previous step in plane opp(I) at x - c_I, or
//                at a wall f*_opp(I)(x), kept in plane I at x.
template <int I, bool WALLS, int MODE>
__device__ __forceinline__ PsmIdx<MODE> src_elem(const LbmArgs& a, const Plan& p) {
    constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
    if constexpr (psm_form(MODE) == PSM_AA_EVEN) return plane_at<MODE>(a, I) + p.cell;
    constexpr int plane_in = psm_form(MODE) == PSM_AA_ODD ? OPP(I) : I;
    constexpr int plane_wall = psm_form(MODE) == PSM_AA_ODD ? I : OPP(I);
    if constexpr (WALLS) {
        bool wx, wy, wz;
        link_walls<I>(p, wx, wy, wz);
        if (wx || wy || wz) return plane_at<MODE>(a, plane_wall) + p.cell;
    }
    // (64-bit: with a periodic wrap the index can pass 2^31 before the plane start is added)
    PsmIdx<MODE> src = (PsmIdx<MODE>)p.cell - a.off[I];
    if (cx == 1) src += p.wxm;
    if (cx == -1) src += p.wxp;
    if (cy == 1) src += p.wym;
    if (cy == -1) src += p.wyp;
    if (cz == 1) src += p.wzm;
    if (cz == -1) src += p.wzp;
    return plane_at<MODE>(a, plane_in) + src;
}


// The two-lattice pull reads an array the kernel does not write (read-only data path);
// the AA pattern reads and writes one array.
template <class SS, int MODE>
__device__ __forceinline__ float ld_pop(const typename SS::T* p) {
    if constexpr (psm_form(MODE) == PSM_AB) return SS::ldg_raw(p);
    else return SS::raw(*p);
}

// Direct pull of direction I of a node, in stored units. GEN: periodic wraps and halfway
// bounce-back with the moving-wall term, from the node's plan; without GEN the caller
// knows that neither occurs for any lane (a node off every lattice face), and the source
// is node - off_I.
template <class SS, int I, bool GEN, int MODE>
__device__ __forceinline__ float pull_one(const LbmArgs& a, const typename SS::T* pin, const Plan& p) {
    if constexpr (!GEN) {
        constexpr int plane_in = psm_form(MODE) == PSM_AA_ODD ? OPP(I) : I;
        PsmIdx<MODE> src = (PsmIdx<MODE>)p.cell;
        if constexpr (psm_form(MODE) != PSM_AA_EVEN) src -= a.off[I];
        return ld_pop<SS, MODE>(pin + (plane_at<MODE>(a, plane_in) + src));
    } else {
        float v = ld_pop<SS, MODE>(pin + src_elem<I, true, MODE>(a, p));
        if constexpr (psm_form(MODE) != PSM_AA_EVEN) {
            bool wx, wy, wz;
            link_walls<I>(p, wx, wy, wz);
            if (wx || wy || wz) v += SS::up(wall_term<I>(a.uw, wx, wy, wz), a.scale);  // moving wall
        }
        return v;
    }
}

template <class SS, bool GEN, int MODE>
__device__ __forceinline__ void pull_all(const LbmArgs& a, const typename SS::T* pin, const Plan& p,
                                         float (&g)[19]) {
    static_for<19>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        g[I] = pull_one<SS, I, GEN, MODE>(a, pin, p);
    });
}

// Shared-memory stage of one z-plane: per direction i a box of TILE_Y rows. A streaming
// step (SHIFT) reads direction i at x - c_i: the boxes of directions with c_x != 0 are
// TILE_X + 2H columns wide from x0 - H (H elements = 16 bytes, so that every box starts
// on a 16-byte boundary, as tensor copies require) and are read at column lane + H - c_x;
// the other boxes, and every box of the in-place AA step, are TILE_X columns from x0.
// Every box is a multiple of 128 bytes, so each one starts 128-byte aligned.
template <int ES, bool SHIFT>
struct Stage {
    static constexpr int H = 16 / ES;
    static constexpr int WB = TILE_X + 2 * H;
    static constexpr bool wide(int i) { return SHIFT && CX(i) != 0; }
    static constexpr int width(int i) { return wide(i) ? WB : TILE_X; }
    static constexpr int slot(int i) { return i == 0 ? 0 : slot(i - 1) + TILE_Y * width(i - 1); }  // elements
    static constexpr int elems = slot(19);
    static constexpr int bytes = elems * ES;
    static_assert((TILE_Y * TILE_X * ES) % 128 == 0 && (TILE_Y * WB * ES) % 128 == 0, "box alignment");
};

// mbarrier and tensor-copy primitives (PTX ISA: mbarrier, cp.async.bulk.tensor).
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Every wait is bounded: after about a quarter of a second at the GB300 clock it counts a
// timeout in the status block (ledds_get_status returns LEDDS_ERR_TIMEOUT) and gives up.
constexpr long long PSM_WAIT_CYCLES = 1ll << 29;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity, DevStatus* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > PSM_WAIT_CYCLES) {
            atomicAdd(&status->wait_timeout, 1);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Issue the boxes of z-plane z of the tile at (x0, y0) into a stage; one thread. The box
// of direction I comes from plane I (plane opp(I) in the AA pattern's streaming step,
// which keeps f*_I there), shifted by -c_I in a streaming step. Boxes that reach beyond
// the lattice are filled with zeros by the copy engine; the rows and lanes that would
// read them take the direct route.
template <int ES, int MODE>
__device__ __forceinline__ void issue_plane(const PsmMaps& m, uint32_t stage, uint32_t full, int x0, int y0, int z) {
    constexpr bool SHIFT = psm_form(MODE) != PSM_AA_EVEN;
    using G = Stage<ES, SHIFT>;
    mbar_expect_tx(full, (unsigned)G::bytes);
    static_for<19>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        constexpr int plane = psm_form(MODE) == PSM_AA_ODD ? OPP(I) : I;
        const CUtensorMap* map = G::wide(I) ? &m.wide : &m.narrow;
        tma_load_4d(stage + (uint32_t)(G::slot(I) * ES), map, x0 - (G::wide(I) ? G::H : 0),
                    y0 - (SHIFT ? CY(I) : 0), z - (SHIFT ? CZ(I) : 0), plane, full);
    });
}

// A warp's row of the stage: g_I of the lane's node, in stored units.
template <class SS, int MODE>
__device__ __forceinline__ void read_stage(const LbmArgs& a, const unsigned char* stage, int lane, int warp,
                                           float (&g)[19]) {
    using T = typename SS::T;
    constexpr bool SHIFT = psm_form(MODE) != PSM_AA_EVEN;
    using G = Stage<(int)sizeof(T), SHIFT>;
    const T* sb = reinterpret_cast<const T*>(stage);
    const int on = warp * TILE_X + lane;            // narrow boxes
    const int ow = warp * G::WB + lane + G::H;      // wide boxes
    static_for<19>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const T v = G::wide(I) ? sb[G::slot(I) + ow - CX(I)] : sb[G::slot(I) + on];
        g[I] = SS::raw(v);
    });
}

// Lanes at the x ends of the lattice in a row off the y and z faces: the directions with
// c_x != 0 wrap or bounce back; re-pulled directly.
template <class SS, int MODE>
__device__ __forceinline__ void fix_x_ends(const LbmArgs& a, const typename SS::T* pin, const Plan& p,
                                           float (&g)[19]) {
    static_for<19>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        if constexpr (CX(I) != 0) g[I] = pull_one<SS, I, true, MODE>(a, pin, p);
    });
}

// c . v for a lattice vector c with components in {-1, 0, 1} known at compile time (no
// multiplications by 0 or +/-1 left to run time), and c^T Q c for a symmetric Q.
template <int CXv, int CYv, int CZv>
__device__ __forceinline__ float cdot(float x, float y, float z) {
    float r = 0.0f;
    if constexpr (CXv != 0) r = CXv > 0 ? x : -x;
    if constexpr (CYv != 0) r = CXv != 0 ? (CYv > 0 ? r + y : r - y) : (CYv > 0 ? y : -y);
    if constexpr (CZv != 0) r = (CXv != 0 || CYv != 0) ? (CZv > 0 ? r + z : r - z) : (CZv > 0 ? z : -z);
    return r;
}

// Store of the post-collision f*_I(x) by a step of form MODE (WALLS as for src_elem); v
// is in stored units (g times the storage scale):
//   PSM_AB:      plane I at x of the other array;
//   PSM_AA_EVEN: plane opp(I) at x, in place (the next step streams it);
//   PSM_AA_ODD:  pushed to plane I at x + c_I, where the next step reads it in place, or,
//                for a link into a wall, returned to x as f_opp(I) in plane opp(I) with
//                the moving-wall term of that direction (halfway bounce-back).
// `node` points at the node's element of plane 0.
template <class SS, int I, int MODE, bool WALLS>
__device__ __forceinline__ void put(const LbmArgs& a, const Plan& p, typename SS::T* node, float v, bool valid) {
    if constexpr (psm_form(MODE) == PSM_AB) {
        SS::store_if(node + plane_at<MODE>(a, I), v, valid);
    } else if constexpr (psm_form(MODE) == PSM_AA_EVEN) {
        SS::store_if(node + plane_at<MODE>(a, OPP(I)), v, valid);
    } else {
        if (!valid) return;
        constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
        if constexpr (WALLS) {
            bool wx, wy, wz;
            link_walls<OPP(I)>(p, wx, wy, wz);
            if (wx || wy || wz) {
                SS::store_raw(node + plane_at<MODE>(a, OPP(I)),
                              v + SS::up(wall_term<OPP(I)>(a.uw, wx, wy, wz), a.scale));
                return;
            }
        }
        PsmIdx<MODE> d = plane_at<MODE>(a, I) + a.off[I];
        if (cx == 1) d += p.wxp;
        if (cx == -1) d += p.wxm;
        if (cy == 1) d += p.wyp;
        if (cy == -1) d += p.wym;
        if (cz == 1) d += p.wzp;
        if (cz == -1) d += p.wzm;
        SS::store_raw(node + d, v);
    }
}

// ------------------------------------------------------------------------------------
// The PSM collision in coefficient form. With g_i = f_i - t_i, the BGK or TRT collision
// of the fluid part weighted by 1 - B_tot (Eqs. lbePS, TRT), the solid terms
// sum_k B_k Omega^s_{i,k} (Eqs. psm1, bk, btot) and the Guo force term expand, direction
// by direction, into
//   g*_i = al g_i + ga g_ibar + t_i (q0 + c_i . q + c_i^T Q c_i)
// with, for We = (1 - B_tot) w+, Wo = (1 - B_tot) w- (Wo = We for BGK), Bs = sum_k B_k,
// V = sum_k B_k u_k, Y = sum_k B_k u_k u_k^T, Z = sum_k B_k u_k^2, E = We - Bs:
//   al = 1 - (We + Wo)/2 - Bs,   ga = Bs - (We - Wo)/2,
//   q0 = We drho - 1.5 rho (E u^2 + Z),   q = 3 rho ((Wo + Bs) u + V),
//   Q  = 4.5 rho (E u u^T + Y),
// and the force terms -3 fw u.F in q0, 3 fwa F in q, 4.5 fw (u F^T + F u^T) in Q
// (fw = (1 - B_tot)(1 - w+/2), fwa the same with w-). The rest direction reduces to
// (1 - We) g_0 + t_0 q0. (Obtained by writing neq_i = g_i - geq_i, splitting the fluid
// relaxation into the parts even and odd in c, and expanding geq_i(rho, u) -
// geq_i(rho, u_k) in c . u and c . u_k.) A node off every solid has Bs = V = Y = Z = 0.
// Every quantity is kept in stored units (g times the storage scale), so 16-bit values
// are used as loaded and stored as computed.
// ------------------------------------------------------------------------------------
struct Coef {
    float al, ga, q0, qx, qy, qz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz;
};

// Solid sums of a node: Bs, B_tot and V, Y, Z of the coefficient form.
struct SolidTerms {
    float Bs, Btot, Vx, Vy, Vz, Yxx, Yyy, Yzz, Yxy, Yxz, Yyz, Z;
};

template <bool TRT, bool SOLID>
__device__ __forceinline__ void node_coef(const LbmArgs& a, float sc, float drho, float rho, float ux, float uy,
                                          float uz, float usq, const SolidTerms& m, Coef& k) {
    const float Btot = SOLID ? m.Btot : 0.0f, Bs = SOLID ? m.Bs : 0.0f;
    const float fl = sb(1.0f, Btot);  // weight of the fluid part
    const float We = mu(fl, a.omega);
    const float Wo = TRT ? mu(fl, a.omega_m) : We;
    if constexpr (TRT) {
        const float hs = mu(0.5f, ad(We, Wo)), hd = mu(0.5f, sb(We, Wo));
        k.al = sb(sb(1.0f, hs), Bs);
        k.ga = sb(Bs, hd);
    } else {
        k.al = sb(sb(1.0f, We), Bs);
        k.ga = Bs;
    }
    const float E = sb(We, Bs);
    const float rs = mu(rho, sc);
    const float r15 = mu(1.5f, rs), r3 = mu(3.0f, rs), r45 = mu(4.5f, rs);
    const float w3 = mu(r3, ad(Wo, Bs)), e45 = mu(r45, E);
    const float Eu = SOLID ? fm(E, usq, m.Z) : mu(E, usq);
    k.q0 = sb(mu(mu(sc, We), drho), mu(r15, Eu));
    const float ex = mu(e45, ux), ey = mu(e45, uy), ez = mu(e45, uz);
    if constexpr (SOLID) {
        k.qx = fm(w3, ux, mu(r3, m.Vx));
        k.qy = fm(w3, uy, mu(r3, m.Vy));
        k.qz = fm(w3, uz, mu(r3, m.Vz));
        k.Qxx = fm(ex, ux, mu(r45, m.Yxx));
        k.Qyy = fm(ey, uy, mu(r45, m.Yyy));
        k.Qzz = fm(ez, uz, mu(r45, m.Yzz));
        k.Qxy = fm(ex, uy, mu(r45, m.Yxy));
        k.Qxz = fm(ex, uz, mu(r45, m.Yxz));
        k.Qyz = fm(ey, uz, mu(r45, m.Yyz));
    } else {
        k.qx = mu(w3, ux);
        k.qy = mu(w3, uy);
        k.qz = mu(w3, uz);
        k.Qxx = mu(ex, ux);
        k.Qyy = mu(ey, uy);
        k.Qzz = mu(ez, uz);
        k.Qxy = mu(ex, uy);
        k.Qxz = mu(ex, uz);
        k.Qyz = mu(ey, uz);
    }
    if (a.has_force) {  // uniform: Guo forcing, weighted by 1 - B_tot like the fluid part
        const float fw = mu(mu(fl, a.guo_pref), sc);
        const float fwa = TRT ? mu(mu(fl, a.guo_pref_m), sc) : fw;
        const float Fx = a.F[0], Fy = a.F[1], Fz = a.F[2];
        const float fw3 = mu(3.0f, fw), fa3 = mu(3.0f, fwa), f45 = mu(4.5f, fw), f9 = mu(9.0f, fw);
        k.q0 = sb(k.q0, mu(fw3, fm(Fz, uz, fm(Fy, uy, mu(Fx, ux)))));
        k.qx = fm(fa3, Fx, k.qx);
        k.qy = fm(fa3, Fy, k.qy);
        k.qz = fm(fa3, Fz, k.qz);
        k.Qxx = fm(f9, mu(ux, Fx), k.Qxx);
        k.Qyy = fm(f9, mu(uy, Fy), k.Qyy);
        k.Qzz = fm(f9, mu(uz, Fz), k.Qzz);
        k.Qxy = fm(f45, fm(ux, Fy, mu(Fx, uy)), k.Qxy);
        k.Qxz = fm(f45, fm(ux, Fz, mu(Fx, uz)), k.Qxz);
        k.Qyz = fm(f45, fm(uy, Fz, mu(Fy, uz)), k.Qyz);
    }
}

// c . q and c^T Q c for a lattice vector c with components in {-1, 0, 1} known at compile
// time, in a fixed order of explicitly rounded additions.
template <int CXv, int CYv, int CZv>
__device__ __forceinline__ float cq(const Coef& k) {
    float r = 0.0f;
    bool first = true;
    if constexpr (CXv != 0) { r = CXv > 0 ? k.qx : -k.qx; first = false; }
    if constexpr (CYv != 0) { r = first ? (CYv > 0 ? k.qy : -k.qy) : (CYv > 0 ? ad(r, k.qy) : sb(r, k.qy)); first = false; }
    if constexpr (CZv != 0) { r = first ? (CZv > 0 ? k.qz : -k.qz) : (CZv > 0 ? ad(r, k.qz) : sb(r, k.qz)); }
    return r;
}
template <int CXv, int CYv, int CZv>
__device__ __forceinline__ float cqqc(const Coef& k) {
    // q0 + c^T Q c: diagonal terms, then the cross term of the two nonzero components
    float r = k.q0;
    if constexpr (CXv != 0) r = ad(r, k.Qxx);
    if constexpr (CYv != 0) r = ad(r, k.Qyy);
    if constexpr (CZv != 0) r = ad(r, k.Qzz);
    if constexpr (CXv != 0 && CYv != 0) r = CXv * CYv > 0 ? fm(2.0f, k.Qxy, r) : fm(-2.0f, k.Qxy, r);
    if constexpr (CXv != 0 && CZv != 0) r = CXv * CZv > 0 ? fm(2.0f, k.Qxz, r) : fm(-2.0f, k.Qxz, r);
    if constexpr (CYv != 0 && CZv != 0) r = CYv * CZv > 0 ? fm(2.0f, k.Qyz, r) : fm(-2.0f, k.Qyz, r);
    return r;
}

// Collision of every direction of one node and its stores: the rest direction, then the
// nine pairs (I, I+1) with c_{I+1} = -c_I, which share t (q0 + c^T Q c) and flip c . q.
template <class SS, int MODE, bool WALLS>
__device__ __forceinline__ void collide_store(const LbmArgs& a, const float (&G)[19], const Coef& k,
                                              const Plan& p, typename SS::T* node, bool valid) {
    put<SS, 0, MODE, WALLS>(a, p, node, fm(ad(k.al, k.ga), G[0], mu(TW(0), k.q0)), valid);  // al + ga = 1 - We
    static_for<9>([&](auto ic) {
        constexpr int I = 1 + 2 * decltype(ic)::value;
        constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
        constexpr float t = TW(I);
        const float P = mu(t, cqqc<cx, cy, cz>(k));
        const float A = mu(t, cq<cx, cy, cz>(k));
        put<SS, I, MODE, WALLS>(a, p, node, fm(k.al, G[I], fm(k.ga, G[I + 1], ad(P, A))), valid);
        put<SS, I + 1, MODE, WALLS>(a, p, node, fm(k.al, G[I + 1], fm(k.ga, G[I], sb(P, A))), valid);
    });
}

// ------------------------------------------------------------------------------------
// The fused PSM step of one node: moments, solid fractions, PSM collision, store, and
// the hydrodynamic force and torque of each solid (Eqs. forceSF, torqueSF) reduced warp
// -> tile (shared FP32) -> particle (global FP64 atomics).
// ------------------------------------------------------------------------------------
// Node (x, y, z) = tile offset (lane, warp, iz) after its pull: G holds the pulled
// populations in stored units and t its solids (node_solids). Entered by every lane of
// the warp together (the force sums are warp-cooperative); `valid` is false for lanes
// beyond the lattice, wwarp true when some lane of the warp has a wall link. hkey/hacc:
// the running force sum of the solid this lane last met down its column.
template <class SS, bool TRT, int MODE, bool MI>
__device__ __forceinline__ void psm_node(const LbmArgs& a, TileCache& tc, float (&G)[19], const Plan& pl,
                                         bool valid, bool wwarp, const Two& t, int lane, int warp, int iz,
                                         typename SS::T* pout, int& hkey, float (&hacc)[6]) {
    constexpr bool SCALED = sizeof(typename SS::T) == 2;
    const float sc = SCALED ? a.scale : 1.0f;
    // (a lane beyond the lattice computes with the values it read at a clamped position or
    // from zero-filled boxes; its results are not stored and it takes no part in any sum)
    // moments, Eqs. (rho), (momentum); rho = 1 + sum g (pairwise sums for ILP)
    float drho = ad(ad(ad(G[0], ad(G[1], G[2])), ad(ad(G[3], G[4]), ad(G[5], G[6]))),
                    ad(ad(ad(ad(G[7], G[8]), ad(G[9], G[10])), ad(ad(G[11], G[12]), ad(G[13], G[14]))),
                       ad(ad(G[15], G[16]), ad(G[17], G[18]))));
    float jx = ad(ad(ad(sb(G[1], G[2]), sb(G[7], G[8])), ad(sb(G[9], G[10]), sb(G[11], G[12]))), sb(G[13], G[14]));
    float jy = ad(ad(ad(sb(G[3], G[4]), sb(G[7], G[8])), ad(sb(G[10], G[9]), sb(G[15], G[16]))), sb(G[17], G[18]));
    float jz = ad(ad(ad(sb(G[5], G[6]), sb(G[11], G[12])), ad(sb(G[14], G[13]), sb(G[15], G[16]))), sb(G[18], G[17]));
    if constexpr (SCALED) {
        drho = mu(drho, a.inv_scale);
        jx = mu(jx, a.inv_scale);
        jy = mu(jy, a.inv_scale);
        jz = mu(jz, a.inv_scale);
    }
    const float rho = ad(1.0f, drho);
    if (a.has_force) {
        jx = fm(0.5f, a.F[0], jx);
        jy = fm(0.5f, a.F[1], jy);
        jz = fm(0.5f, a.F[2], jz);
    }
    const float inv_rho = __frcp_rn(rho);
    const float ux = mu(jx, inv_rho), uy = mu(jy, inv_rho), uz = mu(jz, inv_rho);
    const float usq = fm(uz, uz, fm(uy, uy, mu(ux, ux)));
    typename SS::T* node = pout + pl.cell;
    Coef k;
    const bool solid = __any_sync(FULL, t.ns > 0);  // uniform
    if (!solid) {
        // no lane of the warp meets a solid at this node: the plain fluid collision, and
        // nothing to add to the held force sums
        SolidTerms m;
        node_coef<TRT, false>(a, sc, drho, rho, ux, uy, uz, usq, m, k);
    } else {
        // Per solid, one after the other (so that one solid's data is live at a time):
        // B_k (Eq. bk) and the surface velocity u_k = v_k + w_k x (x - r_k), its terms in
        // the sums V, Y, Z, and its hydrodynamic force and torque (Eqs. forceSF, torqueSF,
        // which need only rho, u and the solid). Down a column a thread rarely meets a
        // second particle within one tile, so it keeps a running FP32 sum for the first
        // solid and the warp flushes to the tile's FP32 sums (native shared atomics) only
        // when some lane meets a different particle (and at the end of the tile); a second
        // solid in a node (rare) is flushed at once. Tiles add to FP64 totals.
        const bool two = __any_sync(FULL, t.ns > 1);  // uniform
        SolidTerms m;
        {
            SolidAt q;
            q.B = 0.f;
            q.ux = q.uy = q.uz = q.ax = q.ay = q.az = 0.f;
            if (t.ns > 0) solid_at<MI>(a, tc, t.e0, t.b0, lane, warp, iz, q);
            const float vx = mu(q.B, q.ux), vy = mu(q.B, q.uy), vz = mu(q.B, q.uz);
            m.Bs = q.B;
            m.Vx = vx;
            m.Vy = vy;
            m.Vz = vz;
            m.Yxx = mu(vx, q.ux);
            m.Yyy = mu(vy, q.uy);
            m.Yzz = mu(vz, q.uz);
            m.Yxy = mu(vx, q.uy);
            m.Yxz = mu(vx, q.uz);
            m.Yyz = mu(vy, q.uz);
            m.Z = fm(vz, q.uz, fm(vy, q.uy, mu(vx, q.ux)));
            const int key0 = t.ns > 0 ? t.e0 : -1;
            float v0[6];
            solid_force(q, rho, sb(ux, q.ux), sb(uy, q.uy), sb(uz, q.uz), a, v0);
            // invariant: hacc is zero whenever hkey < 0; a node without solid keeps the
            // held sum (the lane may meet the same particle again further down)
            const bool change = hkey >= 0 && key0 >= 0 && key0 != hkey;
            if (__any_sync(FULL, change)) warp_flush<!MI>(tc, change ? hkey : -1, hacc);
            if (change) {
                hkey = -1;
#pragma unroll
                for (int c = 0; c < 6; ++c) hacc[c] = 0.f;
            }
            if (key0 >= 0) {
#pragma unroll
                for (int c = 0; c < 6; ++c) hacc[c] = ad(hacc[c], v0[c]);
                hkey = key0;
            }
        }
        if (two) {
            SolidAt q;
            q.B = 0.f;
            q.ux = q.uy = q.uz = q.ax = q.ay = q.az = 0.f;
            if (t.ns > 1) solid_at<MI>(a, tc, t.e1, t.b1, lane, warp, iz, q);
            const float vx = mu(q.B, q.ux), vy = mu(q.B, q.uy), vz = mu(q.B, q.uz);
            m.Bs = ad(m.Bs, q.B);
            m.Vx = ad(m.Vx, vx);
            m.Vy = ad(m.Vy, vy);
            m.Vz = ad(m.Vz, vz);
            m.Yxx = fm(vx, q.ux, m.Yxx);
            m.Yyy = fm(vy, q.uy, m.Yyy);
            m.Yzz = fm(vz, q.uz, m.Yzz);
            m.Yxy = fm(vx, q.uy, m.Yxy);
            m.Yxz = fm(vx, q.uz, m.Yxz);
            m.Yyz = fm(vy, q.uz, m.Yyz);
            m.Z = fm(vz, q.uz, fm(vy, q.uy, fm(vx, q.ux, m.Z)));
            float v1[6];
            solid_force(q, rho, sb(ux, q.ux), sb(uy, q.uy), sb(uz, q.uz), a, v1);
            warp_flush<!MI>(tc, t.ns > 1 ? t.e1 : -1, v1);
        }
        m.Btot = fminf(m.Bs, 1.0f);
        node_coef<TRT, true>(a, sc, drho, rho, ux, uy, uz, usq, m, k);
    }
    if (psm_form(MODE) == PSM_AA_ODD && wwarp) collide_store<SS, MODE, true>(a, G, k, pl, node, valid);
    else collide_store<SS, MODE, false>(a, G, k, pl, node, valid);
}

// Per storage format and route: resident CTAs per SM the PSM kernel is compiled for (its
// register budget) and, for the staged route, the stages in the ring (planes in flight +
// the one being read). Chosen by timing the variants on GB300.
template <int STORE, bool STAGED>
struct PsmCfg {
    static constexpr bool F32 = STORE == LEDDS_STORE_F32;
    static constexpr int minb = STAGED ? (F32 ? 3 : 3) : 4;
    static constexpr int stages = F32 ? 2 : 3;
};

// Shared memory of the PSM kernel: the tile cache, then (staged route) the full and
// empty barriers of each stage and the stages, 128-byte aligned in the shared window.
template <int STORE, bool STAGED, bool SHIFT>
struct PsmSmem {
    static constexpr int S = PsmCfg<STORE, STAGED>::stages;
    static constexpr size_t bars = (sizeof(TileCache) + 15) & ~(size_t)15;
    static constexpr size_t stages = bars + 2 * S * sizeof(unsigned long long);
    static constexpr size_t bytes =
        STAGED ? stages + 128 + (size_t)S * Stage<(int)storage_bytes_c(STORE), SHIFT>::bytes : sizeof(TileCache);
};

// Node (x, y, z) needs no wrap and no bounce-back on any axis.
__device__ __forceinline__ bool off_faces(const LbmArgs& a, int x, int y, int z) {
    return x > 0 && x < a.nx - 1 && y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1;
}

// Force and torque sums of the tile's particles to their FP64 totals (after a CTA barrier).
__device__ __forceinline__ void tile_sums_out(const LbmArgs& a, const TileCache& tc, int cnt) {
    for (int idx = threadIdx.x; idx < 6 * cnt; idx += blockDim.x) {
        int e = idx / 6, c = idx % 6;
        double v = (double)tc.acc[c][e];
        if (v != 0.0) {
            double* dst = c < 3 ? a.Fh + (long long)c * a.pcap : a.Mh + (long long)(c - 3) * a.pcap;
            atomicAdd(dst + tc_pid(tc, e), v);
        }
    }
}

// One 32x8xTILE_Z tile (bx, by, bz), planes zlo .. zhi-1 of it, direct route: each
// thread loads its node's 19 pulled values from global memory (independent loads, all
// in flight at once).
template <int STORE, bool TRT, int MODE, bool SPHD>
__device__ __forceinline__ void psm_tile_direct(const LbmArgs& a, int bx, int by, int bz, int zlo, int zhi,
                                                unsigned char* psm_smem) {
    using SS = Store<STORE>;
    using T = typename SS::T;
    const T* pin = (const T*)a.pop_in;
    T* pout = (T*)a.pop_out;
    TileCache& tc = *reinterpret_cast<TileCache*>(psm_smem);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int x0 = bx * TILE_X, y0 = by * TILE_Y, z0 = bz * a.tz;
    const int tile = (bz * a.nty + by) * a.ntx + bx;
    const int x = x0 + lane, y = y0 + warp;
    const int cnt = min(a.tile_count[tile], a.tile_cap);
    load_tile(a, tc, tile, cnt, x0, y0, z0);
    __syncthreads();

    int hkey = -1;
    float hacc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int iz = zlo; iz < zhi; ++iz) {
        const int z = z0 + iz;
        if (y >= a.ny || z >= a.nz) continue;  // uniform across the warp
        const bool valid = x < a.nx;
        const unsigned long long mask = cnt ? row_mask<!SPHD>(a, tc, cnt, warp, iz) : 0ull;
        // lanes beyond the lattice read at x = nx - 1 (results discarded)
        const int xr = valid ? x : a.nx - 1;
        const bool gen = psm_form(MODE) != PSM_AA_EVEN && __any_sync(FULL, !off_faces(a, xr, y, z));
        Plan pl;
        if (gen || psm_form(MODE) == PSM_AA_ODD) make_plan(a, xr, y, z, pl);
        else cell_plan(a, xr, y, z, pl);
        const bool wwarp = gen && __any_sync(FULL, valid && pl.bw != 0u);
        // the node's solids (before the loads, so that the search's registers and the
        // pulled values are not live together)
        Two t;
        t.ns = 0;
        t.total = 0;
        if (mask) node_solids<SPHD>(a, tc, mask, lane, warp, iz, x, y, z, valid, t);  // uniform
        if (t.total > 2) atomicAdd(&a.status->solids_overflow, 1);
        float g[19];
        if (gen) pull_all<SS, true, MODE>(a, pin, pl, g);
        else pull_all<SS, false, MODE>(a, pin, pl, g);
        psm_node<SS, TRT, MODE, !SPHD>(a, tc, g, pl, valid, wwarp, t, lane, warp, iz, pout, hkey, hacc);
    }
    warp_flush<SPHD>(tc, hkey, hacc);
    __syncthreads();
    tile_sums_out(a, tc, cnt);
}

// The same tile, staged route. Thread 0 keeps S-1 planes of boxes in flight: before it
// refills a stage it waits until every warp has read the plane held there (the stage's
// empty barrier, one arrival per warp); each warp waits for the plane's boxes (the full
// barrier, completed by the copy engine's byte count), reads its row into registers and
// releases the stage before it collides. Rows on a y or z face of the lattice take the
// direct route; in a tile at an x end, the end lanes re-pull their x-shifted directions.
template <int STORE, bool TRT, int MODE, bool SPHD>
__device__ __forceinline__ void psm_tile_staged(const LbmArgs& a, const PsmMaps& m, int bx, int by, int bz,
                                                int zlo, int zhi, unsigned char* psm_smem) {
    using SS = Store<STORE>;
    using T = typename SS::T;
    constexpr int ES = (int)sizeof(T);
    constexpr bool SHIFT = psm_form(MODE) != PSM_AA_EVEN;
    using G = Stage<ES, SHIFT>;
    using SM = PsmSmem<STORE, true, SHIFT>;
    constexpr int S = SM::S;
    const T* pin = (const T*)a.pop_in;
    T* pout = (T*)a.pop_out;
    TileCache& tc = *reinterpret_cast<TileCache*>(psm_smem);
    const uint32_t bar0 = smem_addr(psm_smem + SM::bars);  // full[s] at bar0 + 8 s, empty[s] at + 8 (S + s)
    uint32_t st0 = smem_addr(psm_smem + SM::stages);
    const uint32_t pad = (128u - (st0 & 127u)) & 127u;
    st0 += pad;
    const unsigned char* stg = psm_smem + SM::stages + pad;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int x0 = bx * TILE_X, y0 = by * TILE_Y, z0 = bz * a.tz;
    const int tile = (bz * a.nty + by) * a.ntx + bx;
    const int x = x0 + lane, y = y0 + warp;
    const int nplanes = min(zhi, a.nz - z0) - zlo;  // CTA-uniform
    if (nplanes <= 0) return;
    const bool xend = SHIFT && (x0 == 0 || x0 + TILE_X >= a.nx);  // CTA-uniform

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(bar0 + 8u * s, 1u);
            mbar_init(bar0 + 8u * (S + s), (unsigned)TILE_Y);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int q = 0; q < S - 1 && q < nplanes; ++q)
            issue_plane<ES, MODE>(m, st0 + (uint32_t)(q * G::bytes), bar0 + 8u * q, x0, y0, z0 + zlo + q);
    const int cnt = min(a.tile_count[tile], a.tile_cap);
    load_tile(a, tc, tile, cnt, x0, y0, z0);
    __syncthreads();

    int issued = min(S - 1, nplanes);  // thread 0 only
    bool ok = true;
    int hkey = -1;
    float hacc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int r = 0;
    for (; r < nplanes; ++r) {
        const int s = r % S;
        if (tid == 0 && ok && issued < nplanes) {
            const int q = issued;  // = r + S - 1
            const int sq = q % S;
            if (q >= S) ok = mbar_wait(bar0 + 8u * (S + sq), (unsigned)((q / S - 1) & 1), a.status);
            if (ok) {
                issue_plane<ES, MODE>(m, st0 + (uint32_t)(sq * G::bytes), bar0 + 8u * sq, x0, y0, z0 + zlo + q);
                ++issued;
            }
        }
        const int iz = zlo + r, z = z0 + iz;
        const bool valid = x < a.nx;
        const bool row = y < a.ny;  // uniform
        // the node's solids (from the tile cache) while the plane's boxes are in flight
        Two t;
        t.ns = 0;
        t.total = 0;
        if (row && cnt) {
            const unsigned long long mask = row_mask<!SPHD>(a, tc, cnt, warp, iz);
            if (mask) node_solids<SPHD>(a, tc, mask, lane, warp, iz, x, y, z, valid, t);  // uniform
            if (t.total > 2) atomicAdd(&a.status->solids_overflow, 1);
        }
        const bool landed = __all_sync(FULL, mbar_wait(bar0 + 8u * s, (unsigned)((r / S) & 1), a.status));
        if (!landed) break;  // uniform across the warp
        const bool face = SHIFT && (y == 0 || y == a.ny - 1 || z == 0 || z == a.nz - 1);  // uniform
        float g[19];
        if (row && !face) read_stage<SS, MODE>(a, stg + (size_t)s * G::bytes, lane, warp, g);
        __syncwarp();
        if (lane == 0) mbar_arrive(bar0 + 8u * (S + s));
        if (!row) continue;
        const int xr = valid ? x : a.nx - 1;
        Plan pl;
        if (face || xend || psm_form(MODE) == PSM_AA_ODD) make_plan(a, xr, y, z, pl);
        else cell_plan(a, xr, y, z, pl);
        if (face) {
            pull_all<SS, true, MODE>(a, pin, pl, g);
        } else if (xend) {
            if (valid && (x == 0 || x == a.nx - 1)) fix_x_ends<SS, MODE>(a, pin, pl, g);
        }
        const bool wwarp = (face || xend) && __any_sync(FULL, valid && pl.bw != 0u);
        psm_node<SS, TRT, MODE, !SPHD>(a, tc, g, pl, valid, wwarp, t, lane, warp, iz, pout, hkey, hacc);
    }
    warp_flush<SPHD>(tc, hkey, hacc);
    if (tid == 0) {
        // after a timeout: wait (bounded) for the copies still in flight into this CTA's
        // shared memory before the CTA ends
        for (int q = r; q < issued; ++q) {
            if (!mbar_wait(bar0 + 8u * (q % S), (unsigned)((q / S) & 1), a.status)) break;
        }
    }
    __syncthreads();
    tile_sums_out(a, tc, cnt);
}

template <int STORE, bool TRT, int MODE, bool STAGED, bool SPHD>
__global__ void __launch_bounds__(PSM_THREADS, PsmCfg<STORE, STAGED>::minb)
    k_psm(const __grid_constant__ LbmArgs a, const __grid_constant__ PsmMaps m) {
    extern __shared__ __align__(128) unsigned char psm_smem[];
    // small lattices: a.zsplit CTAs share a tile, each taking tz / zsplit of its planes
    const int part = blockIdx.z % a.zsplit, per = a.tz / a.zsplit;
    if constexpr (STAGED)
        psm_tile_staged<STORE, TRT, MODE, SPHD>(a, m, blockIdx.x, blockIdx.y, blockIdx.z / a.zsplit, part * per,
                                                part * per + per, psm_smem);
    else
        psm_tile_direct<STORE, TRT, MODE, SPHD>(a, blockIdx.x, blockIdx.y, blockIdx.z / a.zsplit, part * per,
                                                part * per + per, psm_smem);
}

// Host side: launch k_psm in form MODE (its shared-memory size is set on first use), and
// the dispatch over storage format, collision operator, route (staged when maps are
// given) and particle geometry (spheres with distance fractions only and no periodic
// wrap of node-particle offsets, or any; lattices with 64-bit offsets take the general
// form).
template <int STORE, bool TRT, int MODE, bool STAGED, bool SPHD>
static cudaError_t launch_psm_form(const LbmArgs& a, const PsmMaps* m, cudaStream_t s) {
    static bool configured = false;
    constexpr size_t smem = PsmSmem<STORE, STAGED, psm_form(MODE) != PSM_AA_EVEN>::bytes;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_psm<STORE, TRT, MODE, STAGED, SPHD>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    static const PsmMaps none{};
    k_psm<STORE, TRT, MODE, STAGED, SPHD>
        <<<dim3(a.ntx, a.nty, a.ntz * a.zsplit), PSM_THREADS, smem, s>>>(a, m ? *m : none);
    return cudaGetLastError();
}

template <int STORE, bool TRT, int MODE, bool STAGED>
static cudaError_t launch_psm_geom(const LbmArgs& a, const PsmMaps* m, cudaStream_t s) {
    if constexpr (!psm_w64(MODE)) {
        if (!a.subdiv_any && !a.mi[0] && !a.mi[1] && !a.mi[2])
            return launch_psm_form<STORE, TRT, MODE, STAGED, true>(a, m, s);
    }
    return launch_psm_form<STORE, TRT, MODE, STAGED, false>(a, m, s);
}

template <int STORE, bool TRT, int MODE>
static cudaError_t launch_psm_route(const LbmArgs& a, const PsmMaps* m, cudaStream_t s) {
    if (m) return launch_psm_geom<STORE, TRT, MODE, true>(a, m, s);
    return launch_psm_geom<STORE, TRT, MODE, false>(a, m, s);
}

template <int MODE>
static cudaError_t launch_psm_mode(const LbmArgs& a, const PsmMaps* m, int store, cudaStream_t s) {
    if (a.trt) {
        if (store == LEDDS_STORE_F32) return launch_psm_route<LEDDS_STORE_F32, true, MODE>(a, m, s);
        if (store == LEDDS_STORE_F16) return launch_psm_route<LEDDS_STORE_F16, true, MODE>(a, m, s);
        return launch_psm_route<LEDDS_STORE_BF16, true, MODE>(a, m, s);
    }
    if (store == LEDDS_STORE_F32) return launch_psm_route<LEDDS_STORE_F32, false, MODE>(a, m, s);
    if (store == LEDDS_STORE_F16) return launch_psm_route<LEDDS_STORE_F16, false, MODE>(a, m, s);
    return launch_psm_route<LEDDS_STORE_BF16, false, MODE>(a, m, s);
}

}  // namespace ledds
