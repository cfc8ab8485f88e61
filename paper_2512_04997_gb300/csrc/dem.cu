// dem.cu -- DEM kernels of the coupled step (Secs. 2.1, 2.2, 3.2.1, 3.2.2; App. A).
//
// Compiled with -fmad=false: every FP64 expression rounds exactly as written, so the
// contact predicate, the cell keys and the integrator evaluate the documented operation
// order.
//
// Design: the cell list is rebuilt once per fluid step by a counting sort on the cell
// key (one radix digit wide enough for the whole key). Each particle then gathers, from
// the 27 neighbouring cells, every particle within the sum of bounding radii plus a
// skin into a sorted candidate list; contact pairs during the substeps are a subset of
// it while no particle moves more than skin/2 (checked, see skin_violation). A warp per
// particle evaluates its candidate pairs, one per lane, and sums them by a fixed
// butterfly; a pair is always evaluated in canonical order (lower id first), so both
// members compute bit-identical forces and tangential histories and the per-particle
// sums of Table 1 need neither atomics nor a second sort.
#include <math.h>
#include <algorithm>

#include "internal.cuh"

namespace ledds {

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x;
    o[1] = y;
    o[2] = z;
}
__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

__device__ __forceinline__ double stv(const DemArgs& A, const double* st, int comp, int k) {
    return st[(long long)comp * A.P.cap + k];
}
__device__ __forceinline__ void ld3(const DemArgs& A, const double* st, int comp, int k, double o[3]) {
    for (int a = 0; a < 3; ++a) o[a] = st[(long long)(comp + a) * A.P.cap + k];
}

__device__ __forceinline__ double min_image(const DemArgs& A, int a, double d) {
    if (A.per[a]) {
        if (d > 0.5 * A.L[a]) d -= A.L[a];
        else if (d < -0.5 * A.L[a]) d += A.L[a];
    }
    return d;
}

// ------------------------------------------------------------------------------------
// Exclusive scan of uint32 (n <= 4096*4096): out[0..n], out[n] = total.
// ------------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 1024, SCAN_ITEMS = 4, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    uint32_t prefix = warp ? warp_sums[warp - 1] : 0u;
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    uint32_t r = prefix + x - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const uint32_t* in, int n, uint32_t* partial) {
    long long base = (long long)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        long long i = base + (long long)threadIdx.x * SCAN_ITEMS + q;
        if (i < n) s += in[i];
    }
    uint32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_scan_partials(uint32_t* partial, int nb) {
    uint32_t v[SCAN_ITEMS], s = 0;
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        int i = threadIdx.x * SCAN_ITEMS + q;
        v[q] = i < nb ? partial[i] : 0u;
        s += v[q];
    }
    uint32_t run = block_exclusive_scan(s, nullptr);
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        int i = threadIdx.x * SCAN_ITEMS + q;
        if (i < nb) partial[i] = run;
        run += v[q];
    }
}

__global__ void k_scan_apply(const uint32_t* in, int n, const uint32_t* partial, uint32_t* out) {
    long long base = (long long)blockIdx.x * SCAN_TILE;
    uint32_t v[SCAN_ITEMS], s = 0;
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        long long i = base + (long long)threadIdx.x * SCAN_ITEMS + q;
        v[q] = i < n ? in[i] : 0u;
        s += v[q];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot) + partial[blockIdx.x];
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        long long i = base + (long long)threadIdx.x * SCAN_ITEMS + q;
        if (i < n) out[i] = run;
        run += v[q];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = run;
}

cudaError_t launch_scan(const uint32_t* in, int n, uint32_t* out, uint32_t* partial, cudaStream_t s) {
    int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb < 1) nb = 1;
    k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(in, n, partial);
    k_scan_partials<<<1, SCAN_THREADS, 0, s>>>(partial, nb);
    k_scan_apply<<<nb, SCAN_THREADS, 0, s>>>(in, n, partial, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Neighbour structure (Sec. 3.2.1): keys, counting sort, candidate lists
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cell_key(const DemArgs& A, const double r[3], int c[3]) {
    for (int a = 0; a < 3; ++a) {
        double q = floor((r[a] - A.lo[a]) / A.gh[a]);
        // clamp before converting: a non-finite position lands in cell 0, never out of range
        int v;
        if (!(q >= 0.0)) v = 0;
        else if (q > A.gn[a] - 1) v = A.gn[a] - 1;
        else v = (int)q;
        c[a] = v;
    }
    return (uint32_t)(c[0] + A.gn[0] * (c[1] + A.gn[1] * c[2]));
}

__global__ void k_keys(DemArgs A, int pst) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.P.n) return;
    double r[3];
    ld3(A, A.P.st[pst], SP, k, r);
    int c[3];
    uint32_t key = cell_key(A, r, c);
    A.keys[k] = key;
    A.rank[k] = (int)atomicAdd(&A.cell_count[key], 1u);
    for (int a = 0; a < 3; ++a) A.P.pos_build[(long long)a * A.P.cap + k] = r[a];
}

__global__ void k_scatter(DemArgs A) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.P.n) return;
    A.sorted_tmp[A.cell_start[A.keys[k]] + A.rank[k]] = k;
}

// ------------------------------------------------------------------------------------
// Ids in ascending order inside each cell, so that the sorted (key, id) list is unique.
// The scatter above places a cell's ids in atomic-arrival order; each cell's segment is
// then ordered from that copy (tmp) into `sorted`: a cell of at most SEG_SMALL ids by one
// thread (insertion sort), a larger one by a CTA that marks its ids in a bitmap over the
// id range (windows of SEG_WIN ids in shared memory) and writes the set bits in order;
// O(ids + n / 32) per large cell, so even a grid of one cell (or every particle in
// cell 0 after a blow-up) is ordered in bounded time.
// ------------------------------------------------------------------------------------
constexpr int SEG_SMALL = 32;
constexpr int SEG_WIN = 1 << 18;
constexpr int SEG_WORDS = SEG_WIN / 32;
constexpr int SEG_THREADS = 1024;
constexpr int SEG_PER_THREAD = SEG_WORDS / SEG_THREADS;
constexpr int SEG_LARGE_CTAS = 64;

// big[0] counts the cells left to the large-cell kernel, listed in big[1 ..]
__global__ void k_segsort_small(const uint32_t* start, int G, const int* tmp, int* sorted, int* big) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G) return;
    int b = (int)start[c], e = (int)start[c + 1];
    if (e - b > SEG_SMALL) {
        big[1 + atomicAdd(&big[0], 1)] = c;
        return;
    }
    for (int i = b; i < e; ++i) {
        int v = tmp[i];
        int j = i - 1;
        while (j >= b && sorted[j] > v) {
            sorted[j + 1] = sorted[j];
            --j;
        }
        sorted[j + 1] = v;
    }
}

__global__ void __launch_bounds__(SEG_THREADS) k_segsort_large(const uint32_t* start, int n, const int* tmp,
                                                               int* sorted, const int* big) {
    __shared__ uint32_t bits[SEG_WORDS];
    __shared__ int warp_sum[SEG_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nbig = big[0];
    for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
        const int c = big[1 + q];
        const int b = (int)start[c], e = (int)start[c + 1];
        int out = b;
        for (int w0 = 0; w0 < n; w0 += SEG_WIN) {
            for (int i = t; i < SEG_WORDS; i += SEG_THREADS) bits[i] = 0u;
            __syncthreads();
            for (int i = b + t; i < e; i += SEG_THREADS) {
                const unsigned r = (unsigned)(tmp[i] - w0);
                if (r < (unsigned)SEG_WIN) atomicOr(&bits[r >> 5], 1u << (r & 31u));
            }
            __syncthreads();
            // thread t owns words t*SEG_PER_THREAD ..: exclusive scan of their bit counts
            uint32_t wv[SEG_PER_THREAD];
            int cnt = 0;
            for (int k = 0; k < SEG_PER_THREAD; ++k) {
                wv[k] = bits[t * SEG_PER_THREAD + k];
                cnt += __popc(wv[k]);
            }
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) warp_sum[warp] = incl;
            __syncthreads();
            int before = 0, total = 0;
            for (int w = 0; w < SEG_THREADS / 32; ++w) {
                const int v = warp_sum[w];
                before += w < warp ? v : 0;
                total += v;
            }
            int pos = out + before + incl - cnt;
            for (int k = 0; k < SEG_PER_THREAD; ++k) {
                uint32_t m = wv[k];
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1u;
                    sorted[pos++] = w0 + (t * SEG_PER_THREAD + k) * 32 + bit;
                }
            }
            out += total;
            __syncthreads();  // bits and warp_sum are reused
        }
    }
}

// Orders every cell segment of the counting sort: tmp (scatter order) -> sorted. big
// holds 2 + n / SEG_SMALL ints; its counter is cleared here.
cudaError_t launch_segsort(const uint32_t* start, int G, int n, const int* tmp, int* sorted, int* big,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(big, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_segsort_small<<<(G + 127) / 128, 128, 0, s>>>(start, G, tmp, sorted, big);
    k_segsort_large<<<SEG_LARGE_CTAS, SEG_THREADS, 0, s>>>(start, n, tmp, sorted, big);
    return cudaGetLastError();
}

// Candidate list of particle i (ascending ids) and its tangential history carried over
// from the previous list (Sec. 3.2.2: look-up in the previous sorted list). One warp per
// particle: lane l < 27 scans neighbour cell l (a cell reached twice on a small periodic
// grid is scanned by its lowest lane only), hits are compacted by ballot into the warp's
// shared list, each entry is placed by its rank (ids are distinct), and finds its history
// by binary search in the previous list.
constexpr int CAND_WARPS = 4;

__global__ void __launch_bounds__(32 * CAND_WARPS) k_candidates(DemArgs A, int ob, int nbuf, int pst) {
    __shared__ int s_list[CAND_WARPS][MAX_CAND_CAP];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int i = blockIdx.x * CAND_WARPS + wib;
    if (i >= A.P.n) return;  // uniform across the warp
    int* list = s_list[wib];
    const double* st = A.P.st[pst];
    double ri[3];
    ld3(A, st, SP, i, ri);
    const double bi = A.P.bound[i];
    const uint32_t key = A.keys[i];
    const int c0 = (int)(key % (uint32_t)A.gn[0]);
    const int c1 = (int)((key / (uint32_t)A.gn[0]) % (uint32_t)A.gn[1]);
    const int c2 = (int)(key / ((uint32_t)A.gn[0] * (uint32_t)A.gn[1]));
    int h = -1;
    if (lane < 27) {
        int q[3] = {c0 + lane % 3 - 1, c1 + (lane / 3) % 3 - 1, c2 + lane / 9 - 1};
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            if (q[a] < 0 || q[a] >= A.gn[a]) {
                if (A.per[a]) q[a] = (q[a] + A.gn[a]) % A.gn[a];
                else ok = false;
            }
        }
        if (ok) h = q[0] + A.gn[0] * (q[1] + A.gn[1] * q[2]);
    }
    const unsigned same = __match_any_sync(0xffffffffu, h);
    if (h >= 0 && __ffs(same) - 1 != lane) h = -1;
    uint32_t s = 0, e = 0;
    if (h >= 0) {
        s = A.cell_start[h];
        e = A.cell_start[h + 1];
    }
    int cnt = 0;
    const unsigned lower = (1u << lane) - 1u;
    while (__any_sync(0xffffffffu, s < e)) {
        bool hit = false;
        int j = -1;
        if (s < e) {
            j = A.sorted[s++];
            if (j != i) {
                double d[3];
                for (int a = 0; a < 3; ++a) d[a] = min_image(A, a, ri[a] - stv(A, st, SP + a, j));
                double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double lim = bi + A.P.bound[j] + A.skin;
                hit = d2 < lim * lim;
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, hit);
        const int pos = cnt + __popc(b & lower);
        if (hit && pos < A.ccap) list[pos] = j;
        cnt += __popc(b);
    }
    if (cnt > A.ccap) {
        if (lane == 0) atomicAdd(&A.status->cand_overflow, 1);
        cnt = A.ccap;
    }
    __syncwarp();
    const int* oc = A.cand[ob] + (long long)i * A.ccap;
    const double* oh = A.hist[ob] + (long long)i * A.ccap * 3;
    int* nc = A.cand[nbuf] + (long long)i * A.ccap;
    double* nh = A.hist[nbuf] + (long long)i * A.ccap * 3;
    const int nold = A.ncand[ob][i];
    for (int m = lane; m < cnt; m += 32) {
        const int v = list[m];
        int r = 0;
        for (int q = 0; q < cnt; ++q) r += list[q] < v;
        nc[r] = v;
        int lo = 0, hi = nold;  // first old entry >= v
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (oc[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        const bool found = lo < nold && oc[lo] == v;
        for (int a = 0; a < 3; ++a) nh[3 * r + a] = found ? oh[3 * lo + a] : 0.0;
    }
    if (lane == 0) A.ncand[nbuf][i] = cnt;
}

// ------------------------------------------------------------------------------------
// Contact geometry
// ------------------------------------------------------------------------------------
struct Geo {
    double delta;
    double en[3];              // unit normal from b to a
    double rca[3], rcb[3];     // arms from the centres to the contact point
    double Ra, Rb;             // radii (spheres) / curvature radii (ellipsoids)
    bool sphere;
};

__device__ __forceinline__ void tri_of(const DemArgs& A, const double* st, int k, double R[9]) {
    for (int m = 0; m < 9; ++m) R[m] = st[(long long)(ST + m) * A.P.cap + k];
}
__device__ __forceinline__ void to_body(const double R[9], const double v[3], double o[3]) {
    for (int m = 0; m < 3; ++m) o[m] = R[3 * m] * v[0] + R[3 * m + 1] * v[1] + R[3 * m + 2] * v[2];
}
__device__ __forceinline__ void to_world(const double R[9], const double b[3], double o[3]) {
    for (int a = 0; a < 3; ++a) o[a] = b[0] * R[a] + b[1] * R[3 + a] + b[2] * R[6 + a];
}

// normal, curvature radius of Eq. (local-curvature), osculating centre at surface point p
__device__ void osc(const double r[3], const double R[9], const double s[3], const double p[3],
                    double* rho, double o[3]) {
    double rel[3] = {p[0] - r[0], p[1] - r[1], p[2] - r[2]};
    double pb[3], nb[3], n[3];
    to_body(R, rel, pb);
    for (int m = 0; m < 3; ++m) nb[m] = pb[m] / (s[m] * s[m]);
    double nn = norm3(nb);
    for (int m = 0; m < 3; ++m) nb[m] /= nn;
    to_world(R, nb, n);
    double a = s[0], b = s[1], c = s[2];
    *rho = b * c * pb[0] * pb[0] / (a * a * a) + a * c * pb[1] * pb[1] / (b * b * b) +
           a * b * pb[2] * pb[2] / (c * c * c);
    for (int m = 0; m < 3; ++m) o[m] = p[m] - (*rho) * n[m];
}

// far intersection (largest parameter) of the line origin + t dir with the ellipsoid
__device__ bool hit(const double r[3], const double R[9], const double s[3], const double org[3],
                    const double dir[3], double* t) {
    double rel[3] = {org[0] - r[0], org[1] - r[1], org[2] - r[2]};
    double q[3], w[3];
    to_body(R, rel, q);
    to_body(R, dir, w);
    double Aq = 0, Bq = 0, Cq = -1.0;
    for (int m = 0; m < 3; ++m) {
        Aq += (w[m] / s[m]) * (w[m] / s[m]);
        Bq += q[m] * w[m] / (s[m] * s[m]);
        Cq += (q[m] / s[m]) * (q[m] / s[m]);
    }
    double disc = Bq * Bq - Aq * Cq;
    if (disc < 0.0 || Aq <= 0.0) return false;
    *t = (-Bq + sqrt(disc)) / Aq;
    return true;
}

// Common-normal iteration with osculating spheres (Sec. 2.1): start on the centre line;
// move each point half way towards the intersection of its ellipsoid with the line
// joining the osculating centres and project it back along the ray from its centre;
// stop when both undamped steps fall below tol * smallest semi-axis.
__device__ __noinline__ bool ell_geo(const DemArgs& A, const double ra[3], const double Ra_[9],
                        const double sa[3], const double rb[3], const double Rb_[9],
                        const double sb[3], Geo& g) {
    double d[3] = {rb[0] - ra[0], rb[1] - ra[1], rb[2] - ra[2]};
    double dn = norm3(d);
    if (dn <= 0.0) return false;
    double u[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
    double mu[3] = {-u[0], -u[1], -u[2]};
    double t, pa[3], pb[3];
    if (!hit(ra, Ra_, sa, ra, u, &t)) return false;
    for (int a = 0; a < 3; ++a) pa[a] = ra[a] + t * u[a];
    if (!hit(rb, Rb_, sb, rb, mu, &t)) return false;
    for (int a = 0; a < 3; ++a) pb[a] = rb[a] + t * mu[a];
    double smin = sa[0];
    for (int m = 0; m < 3; ++m) {
        smin = fmin(smin, sa[m]);
        smin = fmin(smin, sb[m]);
    }
    bool conv = false;
    double oa[3], ob[3], rhoa, rhob;
    for (int it = 0; it < A.ell_max_iter; ++it) {
        osc(ra, Ra_, sa, pa, &rhoa, oa);
        osc(rb, Rb_, sb, pb, &rhob, ob);
        double w[3] = {ob[0] - oa[0], ob[1] - oa[1], ob[2] - oa[2]};
        double wn = norm3(w);
        if (wn <= 0.0) break;
        for (int a = 0; a < 3; ++a) w[a] /= wn;
        double mw[3] = {-w[0], -w[1], -w[2]};
        double ta, tb;
        if (!hit(ra, Ra_, sa, oa, w, &ta)) break;
        if (!hit(rb, Rb_, sb, ob, mw, &tb)) break;
        double da[3], db[3];
        for (int a = 0; a < 3; ++a) {
            da[a] = (oa[a] + ta * w[a]) - pa[a];
            db[a] = (ob[a] + tb * mw[a]) - pb[a];
        }
        double mv = fmax(norm3(da), norm3(db));
        double qa[3], qb[3];
        for (int a = 0; a < 3; ++a) {
            qa[a] = (pa[a] + 0.5 * da[a]) - ra[a];
            qb[a] = (pb[a] + 0.5 * db[a]) - rb[a];
        }
        double qan = norm3(qa), qbn = norm3(qb);
        for (int a = 0; a < 3; ++a) {
            qa[a] /= qan;
            qb[a] /= qbn;
        }
        if (!hit(ra, Ra_, sa, ra, qa, &ta)) break;
        if (!hit(rb, Rb_, sb, rb, qb, &tb)) break;
        for (int a = 0; a < 3; ++a) {
            pa[a] = ra[a] + ta * qa[a];
            pb[a] = rb[a] + tb * qb[a];
        }
        if (mv < A.ell_tol * smin) {
            conv = true;
            break;
        }
    }
    if (!conv) atomicAdd(&A.status->ell_nonconverged, 1);
    osc(ra, Ra_, sa, pa, &rhoa, oa);
    osc(rb, Rb_, sb, pb, &rhob, ob);
    double gv[3] = {oa[0] - ob[0], oa[1] - ob[1], oa[2] - ob[2]};
    double gn = norm3(gv);
    g.delta = rhoa + rhob - gn;
    for (int a = 0; a < 3; ++a) {
        g.en[a] = gv[a] / gn;
        double cp = 0.5 * (pa[a] + pb[a]);
        g.rca[a] = cp - ra[a];
        g.rcb[a] = cp - rb[a];
    }
    g.Ra = rhoa;
    g.Rb = rhob;
    g.sphere = false;
    return true;
}

// Perram-Wertheim separation certificate: with M = R^T diag(s^2) R per ellipsoid (R rows
// = body axes) and d = r_b - r_a, F(l) = l (1 - l) d^T C(l)^-1 d, C(l) = (1 - l) M_a + l M_b;
// the ellipsoids are disjoint if F(l) > 1 for some l (Perram & Wertheim 1985). F is
// evaluated at up to 16 points of a golden-section search for its maximum on [0, 1]
// (C^-1 d by the adjugate); a value above 1 + 1e-9 proves separation. The arithmetic is
// that of the FP64 reference, in the same order.
__device__ __forceinline__ void pw_shape(const double R[9], const double s[3], double M[6]) {
    const double q0 = s[0] * s[0], q1 = s[1] * s[1], q2 = s[2] * s[2];
    M[0] = q0 * R[0] * R[0] + q1 * R[3] * R[3] + q2 * R[6] * R[6];
    M[1] = q0 * R[1] * R[1] + q1 * R[4] * R[4] + q2 * R[7] * R[7];
    M[2] = q0 * R[2] * R[2] + q1 * R[5] * R[5] + q2 * R[8] * R[8];
    M[3] = q0 * R[0] * R[1] + q1 * R[3] * R[4] + q2 * R[6] * R[7];
    M[4] = q0 * R[0] * R[2] + q1 * R[3] * R[5] + q2 * R[6] * R[8];
    M[5] = q0 * R[1] * R[2] + q1 * R[4] * R[5] + q2 * R[7] * R[8];
}
__device__ __forceinline__ double pw_value(const double Ma[6], const double Mb[6], const double d[3], double l) {
    double c[6];
    for (int k = 0; k < 6; ++k) c[k] = (1.0 - l) * Ma[k] + l * Mb[k];
    const double a00 = c[1] * c[2] - c[5] * c[5];
    const double a11 = c[0] * c[2] - c[4] * c[4];
    const double a22 = c[0] * c[1] - c[3] * c[3];
    const double a01 = c[4] * c[5] - c[3] * c[2];
    const double a02 = c[3] * c[5] - c[4] * c[1];
    const double a12 = c[3] * c[4] - c[0] * c[5];
    const double det = c[0] * a00 + c[3] * a01 + c[4] * a02;
    const double q = d[0] * (a00 * d[0] + a01 * d[1] + a02 * d[2]) + d[1] * (a01 * d[0] + a11 * d[1] + a12 * d[2]) +
                     d[2] * (a02 * d[0] + a12 * d[1] + a22 * d[2]);
    return l * (1.0 - l) * q / det;
}
__device__ __noinline__ bool pw_separated(const double ra[3], const double Ra_[9], const double sa[3],
                                          const double rb[3], const double Rb_[9], const double sb[3]) {
    const double margin = 1.0 + 1e-9, gr = 0.6180339887498949;
    double Ma[6], Mb[6], d[3];
    pw_shape(Ra_, sa, Ma);
    pw_shape(Rb_, sb, Mb);
    for (int a = 0; a < 3; ++a) d[a] = rb[a] - ra[a];
    double lo = 0.0, hi = 1.0;
    double c = hi - gr * (hi - lo), e = lo + gr * (hi - lo);
    double Fc = pw_value(Ma, Mb, d, c), Fe = pw_value(Ma, Mb, d, e);
    if (Fc > margin || Fe > margin) return true;
    for (int k = 0; k < 14; ++k) {
        if (Fc > Fe) {
            hi = e;
            e = c;
            Fe = Fc;
            c = hi - gr * (hi - lo);
            Fc = pw_value(Ma, Mb, d, c);
            if (Fc > margin) return true;
        } else {
            lo = c;
            c = e;
            Fc = Fe;
            e = lo + gr * (hi - lo);
            Fe = pw_value(Ma, Mb, d, e);
            if (Fe > margin) return true;
        }
    }
    return false;
}

// Geometry of the canonical pair (a < b) from state buffer st; false if no contact.
__device__ bool pair_geo(const DemArgs& A, const double* st, int a, int b, Geo& g) {
    double dd[3];
    for (int c = 0; c < 3; ++c) dd[c] = min_image(A, c, stv(A, st, SP + c, a) - stv(A, st, SP + c, b));
    const int sha = A.P.shape[a], shb = A.P.shape[b];
    if (sha == LEDDS_SPHERE && shb == LEDDS_SPHERE) {
        double d2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
        double dist = sqrt(d2);
        double Ra = A.P.radius[a], Rb = A.P.radius[b];
        g.delta = (Ra + Rb) - dist;
        if (!(g.delta > 0.0)) return false;
        for (int c = 0; c < 3; ++c) {
            g.en[c] = dd[c] / dist;
            g.rca[c] = -Ra * g.en[c];
            g.rcb[c] = Rb * g.en[c];
        }
        g.Ra = Ra;
        g.Rb = Rb;
        g.sphere = true;
        return true;
    }
    double dist = norm3(dd);
    if (!((A.P.bound[a] + A.P.bound[b]) - dist > 0.0)) return false;
    // Screens (ell_screen, on by default): two exact tests of disjointness before the
    // common-normal iteration; a pair either rejects is disjoint, so the iteration does not
    // run for it (the iteration can fail to converge on such near-tangent pairs and then
    // report a spurious overlap). Off: the iteration alone decides, as Sec. 2.1 states.
    if (A.ell_screen) {   // separating plane across the centre line: supports |diag(s) R n|
        // that do not reach across the centre distance mean no contact
        double n[3], h[2];
        for (int c = 0; c < 3; ++c) n[c] = dd[c] / dist;
        for (int k = 0; k < 2; ++k) {
            const int q = k == 0 ? a : b;
            double t = 0.0;
            for (int m = 0; m < 3; ++m) {
                double bm = stv(A, st, ST + 3 * m, q) * n[0] + stv(A, st, ST + 3 * m + 1, q) * n[1] +
                            stv(A, st, ST + 3 * m + 2, q) * n[2];
                double v = A.P.semi[(long long)m * A.P.cap + q] * bm;
                t = t + v * v;
            }
            h[k] = sqrt(t);
        }
        if ((h[0] + h[1]) < dist * (1.0 - 1e-12)) return false;
    }
    double ra[3], rb[3], Ra_[9], Rb_[9], sa[3], sb[3];
    for (int c = 0; c < 3; ++c) {
        ra[c] = stv(A, st, SP + c, a);
        rb[c] = ra[c] - dd[c];
        sa[c] = A.P.semi[(long long)c * A.P.cap + a];
        sb[c] = A.P.semi[(long long)c * A.P.cap + b];
    }
    tri_of(A, st, a, Ra_);
    tri_of(A, st, b, Rb_);
    if (A.ell_screen && pw_separated(ra, Ra_, sa, rb, Rb_, sb)) return false;  // proven disjoint
    if (!ell_geo(A, ra, Ra_, sa, rb, Rb_, sb, g)) return false;
    return g.delta > 0.0;
}

// Particle-wall geometry, face = 2*axis + side: a static plane with inward normal at the
// halfway position, surface velocity u_w; infinite mass and radius.
__device__ __noinline__ bool wall_geo(const DemArgs& A, const double* st, int k, int face, Geo& g) {
    int a = face >> 1, side = face & 1;
    double nrm[3] = {0.0, 0.0, 0.0};
    nrm[a] = side == 0 ? 1.0 : -1.0;
    double r[3];
    ld3(A, st, SP, k, r);
    if (A.P.shape[k] == LEDDS_SPHERE) {
        double R = A.P.radius[k];
        double dist = side == 0 ? r[a] - A.lo[a] : A.hi[a] - r[a];
        g.delta = R - dist;
        if (!(g.delta > 0.0)) return false;
        for (int c = 0; c < 3; ++c) {
            g.en[c] = nrm[c];
            g.rca[c] = -R * nrm[c];
            g.rcb[c] = 0.0;
        }
        g.Ra = R;
        g.sphere = true;
        return true;
    }
    double R9[9], s[3];
    tri_of(A, st, k, R9);
    for (int c = 0; c < 3; ++c) s[c] = A.P.semi[(long long)c * A.P.cap + k];
    double nb[3], pb[3], pw[3], p[3];
    to_body(R9, nrm, nb);
    double den = sqrt(s[0] * s[0] * nb[0] * nb[0] + s[1] * s[1] * nb[1] * nb[1] + s[2] * s[2] * nb[2] * nb[2]);
    for (int m = 0; m < 3; ++m) pb[m] = -s[m] * s[m] * nb[m] / den;
    to_world(R9, pb, pw);
    for (int c = 0; c < 3; ++c) p[c] = r[c] + pw[c];
    double sd = side == 0 ? p[a] - A.lo[a] : A.hi[a] - p[a];
    g.delta = -sd;
    if (!(g.delta > 0.0)) return false;
    double rho, o[3];
    osc(r, R9, s, p, &rho, o);
    for (int c = 0; c < 3; ++c) {
        g.en[c] = nrm[c];
        g.rca[c] = (p[c] + 0.5 * g.delta * nrm[c]) - r[c];
        g.rcb[c] = 0.0;
    }
    g.Ra = rho;
    g.sphere = false;
    return true;
}

// ------------------------------------------------------------------------------------
// Spring-dashpot force on a (Eqs. spring_dashpot_easy, fnScal, trangential-history,
// coulombCoeff; App. A for the Hertz coefficients). h: tangential displacement of the
// canonical pair, updated in place. Ft receives the tangential part.
// ------------------------------------------------------------------------------------
__device__ void spring_dashpot(const DemArgs& A, const Geo& g, double Rstar, double mstar,
                               const double va[3], const double wa[3], const double vb[3],
                               const double wb[3], double h[3], double F[3], double Ft[3]) {
    double kn, kt, gn, gt;
    if (A.law == LEDDS_LAW_LINEAR) {
        kn = A.k_n;
        kt = A.k_t;
        gn = -2.0 * A.beta * sqrt(kn * mstar);
        gt = -2.0 * A.beta * sqrt(kt * mstar);
    } else {
        double sq = sqrt(Rstar * g.delta);
        kn = 4.0 / 3.0 * A.Ystar * sq;
        kt = 8.0 * A.Gstar * sq;
        double Sn = 2.0 * A.Ystar * sq;
        double St = 8.0 * A.Gstar * sq;
        gn = -2.0 * sqrt(5.0 / 6.0) * A.beta * sqrt(Sn * mstar);
        gt = -2.0 * sqrt(5.0 / 6.0) * A.beta * sqrt(St * mstar);
    }
    double ca[3], cb[3], vrel[3];
    cross3(wa, g.rca, ca);
    cross3(wb, g.rcb, cb);
    for (int c = 0; c < 3; ++c) vrel[c] = (va[c] + ca[c]) - (vb[c] + cb[c]);
    double vn = dot3(vrel, g.en);
    double vt[3];
    for (int c = 0; c < 3; ++c) vt[c] = vrel[c] - vn * g.en[c];
    double fn = kn * g.delta - gn * vn;
    double hn = dot3(h, g.en);
    double hp[3];
    for (int c = 0; c < 3; ++c) hp[c] = h[c] - hn * g.en[c];
    double lh = norm3(h), lp = norm3(hp);
    if (lp > 0.0)
        for (int c = 0; c < 3; ++c) hp[c] *= lh / lp;
    for (int c = 0; c < 3; ++c) h[c] = hp[c] + vt[c] * A.dt;
    for (int c = 0; c < 3; ++c) Ft[c] = -kt * h[c] - gt * vt[c];
    double lft = norm3(Ft), lfn = fabs(fn);
    if (lft > A.mu * lfn) {
        double sc = lft > 0.0 ? A.mu * lfn / lft : 0.0;
        for (int c = 0; c < 3; ++c) Ft[c] *= sc;
        if (kt > 0.0)
            for (int c = 0; c < 3; ++c) h[c] = -(Ft[c] + gt * vt[c]) / kt;
    }
    for (int c = 0; c < 3; ++c) F[c] = fn * g.en[c] + Ft[c];
}

// Contribution of candidate slot m of particle i (state buffer st): the canonical pair
// force is applied with the sign of i's membership; the slot's tangential history is
// updated (and reset when the pair is not in contact).
__device__ __noinline__ void pair_contrib(const DemArgs& A, const double* st, int cb, int i, int m, double F[3],
                             double M[3]) {
    const int j = A.cand[cb][(long long)i * A.ccap + m];
    double* hl = A.hist[cb] + ((long long)i * A.ccap + m) * 3;
    const int a = i < j ? i : j, b = i < j ? j : i;
    Geo g;
    if (!pair_geo(A, st, a, b, g)) {
        hl[0] = hl[1] = hl[2] = 0.0;
        return;
    }
    double va[3], wa[3], vb[3], wb[3], h[3], Fp[3], Ft[3];
    ld3(A, st, SV, a, va);
    ld3(A, st, SW, a, wa);
    ld3(A, st, SV, b, vb);
    ld3(A, st, SW, b, wb);
    for (int c = 0; c < 3; ++c) h[c] = hl[c];
    double Rstar = 1.0 / (1.0 / g.Ra + 1.0 / g.Rb);
    double mstar = 1.0 / (1.0 / A.P.mass[a] + 1.0 / A.P.mass[b]);
    spring_dashpot(A, g, Rstar, mstar, va, wa, vb, wb, h, Fp, Ft);
    for (int c = 0; c < 3; ++c) hl[c] = h[c];
    double Mi[3];
    if (g.sphere) {
        // Sec. 2.1: M = -R e_n x F_t for both members
        double mr[3];
        cross3(g.en, Ft, mr);
        double Ri = i == a ? g.Ra : g.Rb;
        for (int c = 0; c < 3; ++c) Mi[c] = -Ri * mr[c];
    } else if (i == a) {
        cross3(g.rca, Fp, Mi);  // Eq. (torque)
    } else {
        double mF[3] = {-Fp[0], -Fp[1], -Fp[2]};
        cross3(g.rcb, mF, Mi);
    }
    double sgn = i == a ? 1.0 : -1.0;
    for (int c = 0; c < 3; ++c) {
        F[c] += sgn * Fp[c];
        M[c] += Mi[c];
    }
}

// Contribution of wall face `face` on particle i (history per particle and face).
__device__ __noinline__ void wall_contrib(const DemArgs& A, const double* st, int i, int face, double F[3], double M[3]) {
    const int ax = face >> 1;
    double* wh = A.whist + ((long long)i * 6 + face) * 3;
    Geo g;
    if (A.per[ax] || !wall_geo(A, st, i, face, g)) {
        wh[0] = wh[1] = wh[2] = 0.0;
        return;
    }
    double vi[3], wi[3];
    ld3(A, st, SV, i, vi);
    ld3(A, st, SW, i, wi);
    const double* uw = A.uw[ax][face & 1];
    double zero[3] = {0.0, 0.0, 0.0}, Fw[3], Ft[3], Mw[3];
    spring_dashpot(A, g, g.Ra, A.P.mass[i], vi, wi, uw, zero, wh, Fw, Ft);
    if (g.sphere) {
        double mr[3];
        cross3(g.en, Ft, mr);
        for (int c = 0; c < 3; ++c) Mw[c] = -g.Ra * mr[c];
    } else {
        cross3(g.rca, Fw, Mw);
    }
    for (int c = 0; c < 3; ++c) {
        F[c] += Fw[c];
        M[c] += Mw[c];
    }
}

// ------------------------------------------------------------------------------------
// FP32 contact arithmetic (force_fp32): positions and velocities are differenced in FP64
// and rounded, the contact predicate is decided in FP64 exactly as in the FP64 path (so
// contact sets do not change), the spring-dashpot force and torque are evaluated in FP32
// and summed per particle in FP64. The tangential history stays stored in FP64.
// ------------------------------------------------------------------------------------
struct GeoF {
    float delta;
    float en[3];
    float rca[3], rcb[3];
    float Ra, Rb;
    bool sphere;
};

__device__ __forceinline__ void cross3f(const float a[3], const float b[3], float o[3]) {
    float x = a[1] * b[2] - a[2] * b[1];
    float y = a[2] * b[0] - a[0] * b[2];
    float z = a[0] * b[1] - a[1] * b[0];
    o[0] = x;
    o[1] = y;
    o[2] = z;
}
__device__ __forceinline__ float dot3f(const float a[3], const float b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ float norm3f(const float a[3]) { return sqrtf(dot3f(a, a)); }

__device__ __forceinline__ void geo_to_f(const Geo& g, GeoF& f) {
    f.delta = (float)g.delta;
    for (int c = 0; c < 3; ++c) {
        f.en[c] = (float)g.en[c];
        f.rca[c] = (float)g.rca[c];
        f.rcb[c] = (float)g.rcb[c];
    }
    f.Ra = (float)g.Ra;
    f.Rb = (float)g.Rb;
    f.sphere = g.sphere;
}

// Sphere pair with dd = r_a - r_b (FP64, minimum image). The FP64 path's predicate
// (Ra + Rb) - sqrt(|dd|^2) > 0 is decided from num = (Ra + Rb)^2 - |dd|^2 whenever |num|
// exceeds its rounding error by far, and exactly as written otherwise; the overlap is
// num / (Ra + Rb + |dd|), free of cancellation.
__device__ __forceinline__ bool sphere_geo_f(const double dd[3], double Ra, double Rb, GeoF& g) {
    const double d2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
    const double S = Ra + Rb;
    const double S2 = S * S;
    const double num = S2 - d2;
    if (fabs(num) <= 1e-10 * S2) {
        if (!((S - sqrt(d2)) > 0.0)) return false;
    } else if (!(num > 0.0)) {
        return false;
    }
    const float dist = sqrtf((float)d2);
    g.delta = (float)num / ((float)S + dist);
    const float inv = 1.0f / dist;
    const float ra = (float)Ra, rb = (float)Rb;
    for (int c = 0; c < 3; ++c) {
        g.en[c] = (float)dd[c] * inv;
        g.rca[c] = -ra * g.en[c];
        g.rcb[c] = rb * g.en[c];
    }
    g.Ra = ra;
    g.Rb = rb;
    g.sphere = true;
    return true;
}

// The spring-dashpot law of spring_dashpot in FP32; dv = v_a - v_b (rounded from FP64).
__device__ void spring_dashpot_f(const DemArgs& A, const GeoF& g, float Rstar, float mstar, const float dv[3],
                                 const float wa[3], const float wb[3], float h[3], float F[3], float Ft[3]) {
    float kn, kt, gn, gt;
    const float beta = (float)A.beta;
    if (A.law == LEDDS_LAW_LINEAR) {
        kn = (float)A.k_n;
        kt = (float)A.k_t;
        gn = -2.0f * beta * sqrtf(kn * mstar);
        gt = -2.0f * beta * sqrtf(kt * mstar);
    } else {
        const float sq = sqrtf(Rstar * g.delta);
        const float Ys = (float)A.Ystar, Gs = (float)A.Gstar;
        kn = 4.0f / 3.0f * Ys * sq;
        kt = 8.0f * Gs * sq;
        const float Sn = 2.0f * Ys * sq;
        const float St = 8.0f * Gs * sq;
        gn = -2.0f * 0.91287093f * beta * sqrtf(Sn * mstar);   // 0.91287093 = sqrt(5/6)
        gt = -2.0f * 0.91287093f * beta * sqrtf(St * mstar);
    }
    float ca[3], cb[3], vrel[3];
    cross3f(wa, g.rca, ca);
    cross3f(wb, g.rcb, cb);
    for (int c = 0; c < 3; ++c) vrel[c] = dv[c] + (ca[c] - cb[c]);
    const float vn = dot3f(vrel, g.en);
    float vt[3];
    for (int c = 0; c < 3; ++c) vt[c] = vrel[c] - vn * g.en[c];
    const float fn = kn * g.delta - gn * vn;
    const float hn = dot3f(h, g.en);
    float hp[3];
    for (int c = 0; c < 3; ++c) hp[c] = h[c] - hn * g.en[c];
    const float lh = norm3f(h), lp = norm3f(hp);
    if (lp > 0.0f)
        for (int c = 0; c < 3; ++c) hp[c] *= lh / lp;
    const float dt = (float)A.dt;
    for (int c = 0; c < 3; ++c) h[c] = hp[c] + vt[c] * dt;
    for (int c = 0; c < 3; ++c) Ft[c] = -kt * h[c] - gt * vt[c];
    const float lft = norm3f(Ft), lfn = fabsf(fn);
    const float mu = (float)A.mu;
    if (lft > mu * lfn) {
        const float sc = lft > 0.0f ? mu * lfn / lft : 0.0f;
        for (int c = 0; c < 3; ++c) Ft[c] *= sc;
        if (kt > 0.0f)
            for (int c = 0; c < 3; ++c) h[c] = -(Ft[c] + gt * vt[c]) / kt;
    }
    for (int c = 0; c < 3; ++c) F[c] = fn * g.en[c] + Ft[c];
}

// Compensated FP32 sums: a value is the unevaluated pair hi + lo, added with Knuth's
// TwoSum, so sums of FP32 contact forces keep about 48 significant bits (the FP64 sum of
// the same terms to within 2^-48) while running on the FP32 pipes. Converted to FP64 once
// per particle.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    const float hi = __fadd_rn(s, lo);
    return F2{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}
__device__ __forceinline__ F2 f2_add(F2 a, float b) { return f2_add(a, F2{b, 0.0f}); }

// Ellipsoid geometry (FP64) rounded for the FP32 force path; out of line, so that the
// sphere path keeps its registers.
__device__ __noinline__ bool pair_geo_f_general(const DemArgs& A, const double* st, int a, int b, GeoF& g) {
    Geo g64;
    if (!pair_geo(A, st, a, b, g64)) return false;
    geo_to_f(g64, g);
    return true;
}
__device__ __noinline__ bool wall_geo_f_general(const DemArgs& A, const double* st, int i, int face, GeoF& g) {
    Geo g64;
    if (!wall_geo(A, st, i, face, g64)) return false;
    geo_to_f(g64, g);
    return true;
}

// pair_contrib with FP32 contact arithmetic (ellipsoid geometry stays FP64).
template <bool SPHERES>
__device__ void pair_contrib_f(const DemArgs& A, const double* st, int cb, int i, int m, F2 F[3], F2 M[3]) {
    const int j = A.cand[cb][(long long)i * A.ccap + m];
    double* hl = A.hist[cb] + ((long long)i * A.ccap + m) * 3;
    const int a = i < j ? i : j, b = i < j ? j : i;
    GeoF g;
    bool hit_;
    if (SPHERES || (A.P.shape[a] == LEDDS_SPHERE && A.P.shape[b] == LEDDS_SPHERE)) {
        double dd[3];
        for (int c = 0; c < 3; ++c) dd[c] = min_image(A, c, stv(A, st, SP + c, a) - stv(A, st, SP + c, b));
        hit_ = sphere_geo_f(dd, A.P.radius[a], A.P.radius[b], g);
    } else {
        hit_ = pair_geo_f_general(A, st, a, b, g);
    }
    if (!hit_) {
        hl[0] = hl[1] = hl[2] = 0.0;
        return;
    }
    float dv[3], wa[3], wb[3], h[3], Fp[3], Ft[3];
    for (int c = 0; c < 3; ++c) {
        dv[c] = (float)(stv(A, st, SV + c, a) - stv(A, st, SV + c, b));
        wa[c] = (float)stv(A, st, SW + c, a);
        wb[c] = (float)stv(A, st, SW + c, b);
        h[c] = (float)hl[c];
    }
    const float Rstar = g.Ra * g.Rb / (g.Ra + g.Rb);
    const float ma = (float)A.P.mass[a], mb = (float)A.P.mass[b];
    const float mstar = ma * mb / (ma + mb);
    spring_dashpot_f(A, g, Rstar, mstar, dv, wa, wb, h, Fp, Ft);
    for (int c = 0; c < 3; ++c) hl[c] = (double)h[c];
    float Mi[3];
    if (g.sphere) {
        float mr[3];
        cross3f(g.en, Ft, mr);
        const float Ri = i == a ? g.Ra : g.Rb;
        for (int c = 0; c < 3; ++c) Mi[c] = -Ri * mr[c];
    } else if (i == a) {
        cross3f(g.rca, Fp, Mi);
    } else {
        float mF[3] = {-Fp[0], -Fp[1], -Fp[2]};
        cross3f(g.rcb, mF, Mi);
    }
    const float sgn = i == a ? 1.0f : -1.0f;
    for (int c = 0; c < 3; ++c) {
        F[c] = f2_add(F[c], sgn * Fp[c]);
        M[c] = f2_add(M[c], Mi[c]);
    }
}

// wall_contrib with FP32 contact arithmetic.
template <bool SPHERES>
__device__ void wall_contrib_f(const DemArgs& A, const double* st, int i, int face, F2 F[3], F2 M[3]) {
    const int ax = face >> 1, side = face & 1;
    double* wh = A.whist + ((long long)i * 6 + face) * 3;
    if (A.per[ax]) {
        wh[0] = wh[1] = wh[2] = 0.0;
        return;
    }
    GeoF g;
    if (SPHERES || A.P.shape[i] == LEDDS_SPHERE) {
        const double R = A.P.radius[i];
        const double r = stv(A, st, SP + ax, i);
        const double dist = side == 0 ? r - A.lo[ax] : A.hi[ax] - r;
        const double delta = R - dist;
        if (!(delta > 0.0)) {
            wh[0] = wh[1] = wh[2] = 0.0;
            return;
        }
        g.delta = (float)delta;
        const float Rf = (float)R;
        for (int c = 0; c < 3; ++c) {
            g.en[c] = c == ax ? (side == 0 ? 1.0f : -1.0f) : 0.0f;
            g.rca[c] = -Rf * g.en[c];
            g.rcb[c] = 0.0f;
        }
        g.Ra = Rf;
        g.sphere = true;
    } else if (!wall_geo_f_general(A, st, i, face, g)) {
        wh[0] = wh[1] = wh[2] = 0.0;
        return;
    }
    const double* uw = A.uw[ax][side];
    float dv[3], wi[3], h[3], zero[3] = {0.0f, 0.0f, 0.0f}, Fw[3], Ft[3], Mw[3];
    for (int c = 0; c < 3; ++c) {
        dv[c] = (float)(stv(A, st, SV + c, i) - uw[c]);
        wi[c] = (float)stv(A, st, SW + c, i);
        h[c] = (float)wh[c];
    }
    spring_dashpot_f(A, g, g.Ra, (float)A.P.mass[i], dv, wi, zero, h, Fw, Ft);
    for (int c = 0; c < 3; ++c) wh[c] = (double)h[c];
    if (g.sphere) {
        float mr[3];
        cross3f(g.en, Ft, mr);
        for (int c = 0; c < 3; ++c) Mw[c] = -g.Ra * mr[c];
    } else {
        cross3f(g.rca, Fw, Mw);
    }
    for (int c = 0; c < 3; ++c) {
        F[c] = f2_add(F[c], Fw[c]);
        M[c] = f2_add(M[c], Mw[c]);
    }
}

// ------------------------------------------------------------------------------------
// Pair-once evaluation (simulations with ellipsoids, whose common-normal geometry is
// costly): the canonical pairs (i < j) of the candidate lists are listed once per rebuild;
// each substep evaluates every pair once, one thread per pair, and each particle then
// gathers +/-F and its torque. Both members receive exactly opposite forces.
// ------------------------------------------------------------------------------------
// First slot of particle i's (ascending) candidate list whose id exceeds v.
__device__ __forceinline__ int first_above(const int* cl, int nc, int v) {
    int lo = 0, hi = nc;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cl[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_cpair_count(DemArgs A, int cb, uint32_t* cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.P.n) return;
    const int nc = A.ncand[cb][i];
    cnt[i] = (uint32_t)(nc - first_above(A.cand[cb] + (long long)i * A.ccap, nc, i));
}

// pair code = i * MAX_CAND_CAP + slot
__global__ void k_cpair_emit(DemArgs A, int cb, const uint32_t* off, uint32_t* pim) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.P.n) return;
    const int nc = A.ncand[cb][i];
    uint32_t o = off[i];
    for (int m = first_above(A.cand[cb] + (long long)i * A.ccap, nc, i); m < nc; ++m)
        pim[o++] = (uint32_t)i * MAX_CAND_CAP + (uint32_t)m;
}

// Canonical pair (a, slot m of a, partner b > a): force on a and the torques on a and b,
// FP64 contact arithmetic; updates the slot's tangential history. False if no contact.
__device__ bool pair_force_d(const DemArgs& A, const double* st, int cb, int a, int m, double F[3],
                             double Ma[3], double Mb[3]) {
    const int b = A.cand[cb][(long long)a * A.ccap + m];
    double* hl = A.hist[cb] + ((long long)a * A.ccap + m) * 3;
    Geo g;
    if (!pair_geo(A, st, a, b, g)) {
        hl[0] = hl[1] = hl[2] = 0.0;
        return false;
    }
    double va[3], wa[3], vb[3], wb[3], h[3], Ft[3];
    ld3(A, st, SV, a, va);
    ld3(A, st, SW, a, wa);
    ld3(A, st, SV, b, vb);
    ld3(A, st, SW, b, wb);
    for (int c = 0; c < 3; ++c) h[c] = hl[c];
    double Rstar = 1.0 / (1.0 / g.Ra + 1.0 / g.Rb);
    double mstar = 1.0 / (1.0 / A.P.mass[a] + 1.0 / A.P.mass[b]);
    spring_dashpot(A, g, Rstar, mstar, va, wa, vb, wb, h, F, Ft);
    for (int c = 0; c < 3; ++c) hl[c] = h[c];
    if (g.sphere) {
        double mr[3];
        cross3(g.en, Ft, mr);
        for (int c = 0; c < 3; ++c) {
            Ma[c] = -g.Ra * mr[c];
            Mb[c] = -g.Rb * mr[c];
        }
    } else {
        double mF[3] = {-F[0], -F[1], -F[2]};
        cross3(g.rca, F, Ma);
        cross3(g.rcb, mF, Mb);
    }
    return true;
}

// The same with FP32 contact arithmetic.
__device__ bool pair_force_f(const DemArgs& A, const double* st, int cb, int a, int m, float F[3], float Ma[3],
                             float Mb[3]) {
    const int b = A.cand[cb][(long long)a * A.ccap + m];
    double* hl = A.hist[cb] + ((long long)a * A.ccap + m) * 3;
    GeoF g;
    bool hit_;
    if (A.P.shape[a] == LEDDS_SPHERE && A.P.shape[b] == LEDDS_SPHERE) {
        double dd[3];
        for (int c = 0; c < 3; ++c) dd[c] = min_image(A, c, stv(A, st, SP + c, a) - stv(A, st, SP + c, b));
        hit_ = sphere_geo_f(dd, A.P.radius[a], A.P.radius[b], g);
    } else {
        hit_ = pair_geo_f_general(A, st, a, b, g);
    }
    if (!hit_) {
        hl[0] = hl[1] = hl[2] = 0.0;
        return false;
    }
    float dv[3], wa[3], wb[3], h[3], Ft[3];
    for (int c = 0; c < 3; ++c) {
        dv[c] = (float)(stv(A, st, SV + c, a) - stv(A, st, SV + c, b));
        wa[c] = (float)stv(A, st, SW + c, a);
        wb[c] = (float)stv(A, st, SW + c, b);
        h[c] = (float)hl[c];
    }
    const float Rstar = g.Ra * g.Rb / (g.Ra + g.Rb);
    const float ma = (float)A.P.mass[a], mb = (float)A.P.mass[b];
    const float mstar = ma * mb / (ma + mb);
    spring_dashpot_f(A, g, Rstar, mstar, dv, wa, wb, h, F, Ft);
    for (int c = 0; c < 3; ++c) hl[c] = (double)h[c];
    if (g.sphere) {
        float mr[3];
        cross3f(g.en, Ft, mr);
        for (int c = 0; c < 3; ++c) {
            Ma[c] = -g.Ra * mr[c];
            Mb[c] = -g.Rb * mr[c];
        }
    } else {
        float mF[3] = {-F[0], -F[1], -F[2]};
        cross3f(g.rca, F, Ma);
        cross3f(g.rcb, mF, Mb);
    }
    return true;
}

// One thread per canonical pair: results [9][pcap] (F, Ma, Mb), FP32 values with FP32
// contact arithmetic, FP64 values otherwise (a pair out of contact stores zeros).
__global__ void __launch_bounds__(128) k_pair_forces(DemArgs A, int in, int cb, const uint32_t* off,
                                                     const uint32_t* pim, void* res, long long pcap) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= (long long)off[A.P.n]) return;
    const uint32_t code = pim[p];
    const int a = (int)(code / MAX_CAND_CAP), m = (int)(code % MAX_CAND_CAP);
    const double* st = A.P.st[in];
    if (A.force_f32) {
        float F[3] = {0.f, 0.f, 0.f}, Ma[3] = {0.f, 0.f, 0.f}, Mb[3] = {0.f, 0.f, 0.f};
        pair_force_f(A, st, cb, a, m, F, Ma, Mb);
        float* r = static_cast<float*>(res);
        for (int c = 0; c < 3; ++c) {
            r[c * pcap + p] = F[c];
            r[(3 + c) * pcap + p] = Ma[c];
            r[(6 + c) * pcap + p] = Mb[c];
        }
    } else {
        double F[3] = {0.0, 0.0, 0.0}, Ma[3] = {0.0, 0.0, 0.0}, Mb[3] = {0.0, 0.0, 0.0};
        pair_force_d(A, st, cb, a, m, F, Ma, Mb);
        double* r = static_cast<double*>(res);
        for (int c = 0; c < 3; ++c) {
            r[c * pcap + p] = F[c];
            r[(3 + c) * pcap + p] = Ma[c];
            r[(6 + c) * pcap + p] = Mb[c];
        }
    }
}

// Index of particle i's pair with candidate slot q (partner j) in the pair list, or -1
// when j's list does not hold i (possible only after a candidate-list overflow, which
// the status reports; the candidate relation is otherwise symmetric).
__device__ __forceinline__ long long pair_index(const DemArgs& A, int cb, const uint32_t* off, int i, int q,
                                                int j, int first_i, bool* owner) {
    if (j > i) {
        *owner = true;
        return (long long)off[i] + (q - first_i);
    }
    *owner = false;
    const int* lj = A.cand[cb] + (long long)j * A.ccap;
    const int ncj = A.ncand[cb][j];
    const int slot = first_above(lj, ncj, i) - 1;
    if (slot < 0 || lj[slot] != i) return -1;
    return (long long)off[j] + (slot - first_above(lj, ncj, j));
}

// Warp per particle: gather the pair results and the wall contacts (Fc, Mc).
__global__ void __launch_bounds__(128, 6) k_contacts_gather(DemArgs A, int in, int cb, const uint32_t* off,
                                                            const void* res, long long pcap) {
    const int k = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (k >= A.P.n) return;  // uniform across the warp
    const int lane = threadIdx.x & 31;
    const int nc = A.ncand[cb][k];
    const int* cl = A.cand[cb] + (long long)k * A.ccap;
    const int first_k = first_above(cl, nc, k);
    const double* st = A.P.st[in];
    double Fd[3], Md[3];
    if (A.force_f32) {
        const float* r = static_cast<const float*>(res);
        F2 f[3], mo[3];
        for (int c = 0; c < 3; ++c) f[c] = mo[c] = F2{0.0f, 0.0f};
        for (int q = lane; q < nc; q += 32) {
            bool own;
            const long long p = pair_index(A, cb, off, k, q, cl[q], first_k, &own);
            if (p < 0) continue;
            for (int c = 0; c < 3; ++c) {
                const float fv = r[c * pcap + p];
                f[c] = f2_add(f[c], own ? fv : -fv);
                mo[c] = f2_add(mo[c], r[((own ? 3 : 6) + c) * pcap + p]);
            }
        }
        if (lane < 6) wall_contrib_f<false>(A, st, k, lane, f, mo);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                F2 of{__shfl_xor_sync(0xffffffffu, f[c].hi, o), __shfl_xor_sync(0xffffffffu, f[c].lo, o)};
                F2 om{__shfl_xor_sync(0xffffffffu, mo[c].hi, o), __shfl_xor_sync(0xffffffffu, mo[c].lo, o)};
                f[c] = f2_add(f[c], of);
                mo[c] = f2_add(mo[c], om);
            }
        for (int c = 0; c < 3; ++c) {
            Fd[c] = (double)f[c].hi + (double)f[c].lo;
            Md[c] = (double)mo[c].hi + (double)mo[c].lo;
        }
    } else {
        const double* r = static_cast<const double*>(res);
        for (int c = 0; c < 3; ++c) Fd[c] = Md[c] = 0.0;
        for (int q = lane; q < nc; q += 32) {
            bool own;
            const long long p = pair_index(A, cb, off, k, q, cl[q], first_k, &own);
            if (p < 0) continue;
            for (int c = 0; c < 3; ++c) {
                const double fv = r[c * pcap + p];
                Fd[c] += own ? fv : -fv;
                Md[c] += r[((own ? 3 : 6) + c) * pcap + p];
            }
        }
        if (lane < 6) wall_contrib(A, st, k, lane, Fd, Md);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Fd[c] += __shfl_xor_sync(0xffffffffu, Fd[c], o);
                Md[c] += __shfl_xor_sync(0xffffffffu, Md[c], o);
            }
    }
    if (lane != 0) return;
    for (int a = 0; a < 3; ++a) {
        A.P.Fc[(long long)a * A.P.cap + k] = Fd[a];
        A.P.Mc[(long long)a * A.P.cap + k] = Md[a];
    }
}

// Warp-cooperative contact sum of particle i: lane l evaluates candidate slots l, l+32
// and wall face l (l < 6); a fixed butterfly sums the lanes (deterministic order): in
// FP64 with FP64 contact arithmetic, in compensated FP32 pairs (converted to FP64 at the
// end) with FP32 contact arithmetic.
__device__ void contact_sum_warp(const DemArgs& A, const double* st, int cb, int i, double F[3],
                                 double M[3]) {
    const int lane = threadIdx.x & 31;
    const int nc = A.ncand[cb][i];
    if (A.force_f32) {
        F2 f[3], m[3];
        for (int c = 0; c < 3; ++c) f[c] = m[c] = F2{0.0f, 0.0f};
        for (int q = lane; q < nc; q += 32) pair_contrib_f<false>(A, st, cb, i, q, f, m);
        if (lane < 6) wall_contrib_f<false>(A, st, i, lane, f, m);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                F2 of{__shfl_xor_sync(0xffffffffu, f[c].hi, off), __shfl_xor_sync(0xffffffffu, f[c].lo, off)};
                F2 om{__shfl_xor_sync(0xffffffffu, m[c].hi, off), __shfl_xor_sync(0xffffffffu, m[c].lo, off)};
                // the same operand order on both lanes of a butterfly pair keeps them equal
                const bool low = (lane & off) == 0;
                f[c] = low ? f2_add(f[c], of) : f2_add(of, f[c]);
                m[c] = low ? f2_add(m[c], om) : f2_add(om, m[c]);
            }
        for (int c = 0; c < 3; ++c) {
            F[c] = (double)f[c].hi + (double)f[c].lo;
            M[c] = (double)m[c].hi + (double)m[c].lo;
        }
        return;
    }
    for (int c = 0; c < 3; ++c) F[c] = M[c] = 0.0;
    for (int q = lane; q < nc; q += 32) pair_contrib(A, st, cb, i, q, F, M);
    if (lane < 6) wall_contrib(A, st, i, lane, F, M);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            F[c] += __shfl_xor_sync(0xffffffffu, F[c], off);
            M[c] += __shfl_xor_sync(0xffffffffu, M[c], off);
        }
}

// ------------------------------------------------------------------------------------
// Integration (Sec. 2.2)
// ------------------------------------------------------------------------------------
// The integrator runs a long dependent FP64 chain per particle, so it uses fused
// multiply-adds and few divisions (explicit __fma_rn: this file is compiled without
// contraction, which the contact predicate and the cell keys need).
__device__ __forceinline__ void cross3_fma(const double a[3], const double b[3], double o[3]) {
    double x = __fma_rn(a[1], b[2], -(a[2] * b[1]));
    double y = __fma_rn(a[2], b[0], -(a[0] * b[2]));
    double z = __fma_rn(a[0], b[1], -(a[1] * b[0]));
    o[0] = x;
    o[1] = y;
    o[2] = z;
}
__device__ __forceinline__ double dot3_fma(const double a[3], const double b[3]) {
    return __fma_rn(a[0], b[0], __fma_rn(a[1], b[1], a[2] * b[2]));
}

// Quaternion orientation update: the triad (rows d_i = columns of the body-to-world
// rotation) becomes a unit quaternion by Shepperd's method (the largest of 4w^2, 4x^2,
// 4y^2, 4z^2 from the diagonal, the rest from off-diagonal sums and differences), is
// turned on the left by (cos(|w| dt/2), sin(|w| dt/2) w/|w|), i.e. by the angle |w| dt
// about the world axis w exactly, normalised, and written back as a triad.
__device__ void quat_turn(double d[9], const double w[3], double dt) {
    // m[a][i] = d[3 i + a]
    const double m00 = d[0], m11 = d[4], m22 = d[8];
    const double m01 = d[3], m10 = d[1], m02 = d[6], m20 = d[2], m12 = d[7], m21 = d[5];
    const double tr = m00 + m11 + m22;
    double q0, q1, q2, q3;
    if (tr >= m00 && tr >= m11 && tr >= m22) {
        q0 = 0.5 * sqrt(1.0 + tr);
        const double f = 0.25 / q0;
        q1 = (m21 - m12) * f; q2 = (m02 - m20) * f; q3 = (m10 - m01) * f;
    } else if (m00 >= m11 && m00 >= m22) {
        q1 = 0.5 * sqrt(1.0 + m00 - m11 - m22);
        const double f = 0.25 / q1;
        q0 = (m21 - m12) * f; q2 = (m01 + m10) * f; q3 = (m02 + m20) * f;
    } else if (m11 >= m22) {
        q2 = 0.5 * sqrt(1.0 - m00 + m11 - m22);
        const double f = 0.25 / q2;
        q0 = (m02 - m20) * f; q1 = (m01 + m10) * f; q3 = (m12 + m21) * f;
    } else {
        q3 = 0.5 * sqrt(1.0 - m00 - m11 + m22);
        const double f = 0.25 / q3;
        q0 = (m10 - m01) * f; q1 = (m02 + m20) * f; q2 = (m12 + m21) * f;
    }
    const double wn = sqrt(dot3_fma(w, w));
    double c = 1.0, sn = 0.0;
    if (wn > 0.0) {
        sincos(0.5 * dt * wn, &sn, &c);
        sn /= wn;
    }
    const double p1 = sn * w[0], p2 = sn * w[1], p3 = sn * w[2];
    // (c, p) (x) (q0, q): scalar c q0 - p.q, vector c q + q0 p + p x q
    double r0 = c * q0 - (p1 * q1 + p2 * q2 + p3 * q3);
    double r1 = c * q1 + q0 * p1 + (p2 * q3 - p3 * q2);
    double r2 = c * q2 + q0 * p2 + (p3 * q1 - p1 * q3);
    double r3 = c * q3 + q0 * p3 + (p1 * q2 - p2 * q1);
    const double in = rsqrt(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
    r0 *= in; r1 *= in; r2 *= in; r3 *= in;
    // rotation matrix of r, stored by columns as the triad
    d[0] = 1.0 - 2.0 * (r2 * r2 + r3 * r3);
    d[1] = 2.0 * (r1 * r2 + r0 * r3);
    d[2] = 2.0 * (r1 * r3 - r0 * r2);
    d[3] = 2.0 * (r1 * r2 - r0 * r3);
    d[4] = 1.0 - 2.0 * (r1 * r1 + r3 * r3);
    d[5] = 2.0 * (r2 * r3 + r0 * r1);
    d[6] = 2.0 * (r1 * r3 + r0 * r2);
    d[7] = 2.0 * (r2 * r3 - r0 * r1);
    d[8] = 1.0 - 2.0 * (r1 * r1 + r2 * r2);
}

// Predictor: Eq. (advance-r) and the triad update with w(t), then Gram-Schmidt (or,
// with A.quat, quat_turn); positions wrapped on periodic axes; displacement since the
// last rebuild checked.
__device__ void predict(const DemArgs& A, int k, double r[3], const double v[3], const double acc[3],
                        const double w[3], double d[9]) {
    const double dt = A.dt, h2 = dt * dt / 2.0;
    for (int a = 0; a < 3; ++a) r[a] = __fma_rn(h2, acc[a], __fma_rn(dt, v[a], r[a]));
    for (int a = 0; a < 3; ++a)
        if (A.per[a]) {
            // r - L floor((r - lo)/L); the quotient's floor is 0 well inside [lo, lo + L)
            const double q = r[a] - A.lo[a];
            if (q < 0.0 || q >= 0.999999 * A.L[a]) r[a] = r[a] - A.L[a] * floor(q / A.L[a]);
        }
    if (A.quat) {
        quat_turn(d, w, dt);
    } else {
        for (int m = 0; m < 3; ++m) {
            double* dm = d + 3 * m;
            double wxd[3], ds[3], mid[3], wxm[3];
            cross3_fma(w, dm, wxd);
            for (int a = 0; a < 3; ++a) ds[a] = __fma_rn(dt, wxd[a], dm[a]);
            for (int a = 0; a < 3; ++a) mid[a] = 0.5 * (dm[a] + ds[a]);
            cross3_fma(w, mid, wxm);
            for (int a = 0; a < 3; ++a) dm[a] = __fma_rn(dt, wxm[a], dm[a]);
        }
        double* d1 = d;
        double* d2 = d + 3;
        const double i1 = rsqrt(dot3_fma(d1, d1));
        for (int a = 0; a < 3; ++a) d1[a] *= i1;
        const double p = dot3_fma(d2, d1);
        for (int a = 0; a < 3; ++a) d2[a] = __fma_rn(-p, d1[a], d2[a]);
        const double i2 = rsqrt(dot3_fma(d2, d2));
        for (int a = 0; a < 3; ++a) d2[a] *= i2;
        cross3_fma(d1, d2, d + 6);
    }
    double disp2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = min_image(A, a, r[a] - A.P.pos_build[(long long)a * A.P.cap + k]);
        disp2 = __fma_rn(e, e, disp2);
    }
    if (disp2 > 0.25 * A.skin * A.skin) atomicAdd(&A.status->skin_violation, 1);
    bool bad = false;
    for (int a = 0; a < 3; ++a) bad |= !isfinite(r[a]);
    if (bad) atomicAdd(&A.status->nan_detected, 1);
}

// Corrector: a' = F/m + g (1 - rho_f/rho_p); alpha' = R^T I^-1 [R M - (R w) x (I R w)]
// (Eq. advance-omega, body-frame Euler equations), v += dt/2 (a + a'), w += dt/2 (alpha + alpha').
__device__ void correct(const DemArgs& A, int k, const double F[3], const double M[3], const double d[9],
                        double v[3], double w[3]) {
    const double hdt = A.dt / 2.0;
    double an[3], wb[3], Mb[3], Iw[3], gyr[3], ab[3], al[3];
    const double im = 1.0 / A.P.mass[k], gf = A.P.gfac[k];
    for (int a = 0; a < 3; ++a) an[a] = __fma_rn(F[a], im, A.gravity[a] * gf);
    for (int q = 0; q < 3; ++q) {
        wb[q] = dot3_fma(d + 3 * q, w);
        Mb[q] = dot3_fma(d + 3 * q, M);
    }
    double I[3];
    for (int q = 0; q < 3; ++q) I[q] = A.P.inertia[(long long)q * A.P.cap + k];
    const double D = 1.0 / (I[0] * I[1] * I[2]);  // one division for the three inverses
    const double iI[3] = {I[1] * I[2] * D, I[0] * I[2] * D, I[0] * I[1] * D};
    for (int q = 0; q < 3; ++q) Iw[q] = I[q] * wb[q];
    cross3_fma(wb, Iw, gyr);
    for (int q = 0; q < 3; ++q) ab[q] = (Mb[q] - gyr[q]) * iI[q];
    for (int a = 0; a < 3; ++a) al[a] = __fma_rn(ab[0], d[0 + a], __fma_rn(ab[1], d[3 + a], ab[2] * d[6 + a]));
    for (int a = 0; a < 3; ++a) {
        long long o = (long long)a * A.P.cap + k;
        v[a] = __fma_rn(hdt, A.P.acc[o] + an[a], v[a]);
        w[a] = __fma_rn(hdt, A.P.alpha[o] + al[a], w[a]);
        A.P.acc[o] = an[a];
        A.P.alpha[o] = al[a];
    }
}

__device__ __forceinline__ void load_state(const DemArgs& A, const double* st, int k, double r[3],
                                           double v[3], double w[3], double d[9]) {
    ld3(A, st, SP, k, r);
    ld3(A, st, SV, k, v);
    ld3(A, st, SW, k, w);
    tri_of(A, st, k, d);
}
__device__ __forceinline__ void store_state(const DemArgs& A, double* st, int k, const double r[3],
                                            const double v[3], const double w[3], const double d[9]) {
    for (int a = 0; a < 3; ++a) {
        st[(long long)(SP + a) * A.P.cap + k] = r[a];
        st[(long long)(SV + a) * A.P.cap + k] = v[a];
        st[(long long)(SW + a) * A.P.cap + k] = w[a];
    }
    for (int m = 0; m < 9; ++m) st[(long long)(ST + m) * A.P.cap + k] = d[m];
}

// First substep predictor, in place on buffer 0.
__global__ void k_predict_first(DemArgs A) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.P.n) return;
    double r[3], v[3], w[3], d[9], acc[3];
    load_state(A, A.P.st[0], k, r, v, w, d);
    for (int a = 0; a < 3; ++a) acc[a] = A.P.acc[(long long)a * A.P.cap + k];
    predict(A, k, r, v, acc, w, d);
    for (int a = 0; a < 3; ++a) A.P.st[0][(long long)(SP + a) * A.P.cap + k] = r[a];
    for (int m = 0; m < 9; ++m) A.P.st[0][(long long)(ST + m) * A.P.cap + k] = d[m];
}

// End of a substep for one particle (thread per particle): the corrector with the held
// hydrodynamic force, then the predictor of the next substep, from buffer `in` to `out`.
__global__ void k_integrate(DemArgs A, int in, int out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.P.n) return;
    double r[3], v[3], w[3], d[9], Ft[3], Mt[3], acc[3];
    load_state(A, A.P.st[in], k, r, v, w, d);
    for (int a = 0; a < 3; ++a) {
        long long o = (long long)a * A.P.cap + k;
        Ft[a] = A.P.Fc[o] + A.P.Fhp[o];
        Mt[a] = A.P.Mc[o] + A.P.Mhp[o];
    }
    correct(A, k, Ft, Mt, d, v, w);
    for (int a = 0; a < 3; ++a) acc[a] = A.P.acc[(long long)a * A.P.cap + k];
    predict(A, k, r, v, acc, w, d);
    store_state(A, A.P.st[out], k, r, v, w, d);
}

// One DEM substep of a sphere-only simulation with FP32 contact arithmetic in a single
// launch: the contact force and torque of 32 particles (a warp each, lane per candidate,
// compensated FP32 sums reduced by a butterfly and rounded to FP64 once; the sphere-only
// form of k_contacts, without the ellipsoid and FP64 branches, which keeps its registers
// low), then, after a CTA barrier, the corrector of this substep and
// the predictor of the next for the same 32 particles (a lane each, as k_integrate).
// The contacts read only buffer `in` and the integration writes buffer `out`, so the
// CTAs need no ordering among themselves; the launch boundary orders the substeps.
// do_step = 0 (the last substep) computes the contact sums only.
constexpr int SUB_WARPS = 32;  // most warps (particles) per CTA; the launch picks fewer
static_assert(SUB_WARPS <= 32, "the integration phase gives each particle one lane of warp 0");
__global__ void __launch_bounds__(32 * SUB_WARPS, 1) k_substep_spheres(DemArgs A, int in, int out, int cb,
                                                                      int do_step) {
    __shared__ double sF[SUB_WARPS][3], sM[SUB_WARPS][3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;  // particles of this CTA
    const int base = blockIdx.x * wpc;
    const int k = base + w;
    const double* st = A.P.st[in];
    if (k < A.P.n) {  // uniform across the warp
        const int nc = A.ncand[cb][k];
        F2 f[3], m[3];
        for (int c = 0; c < 3; ++c) f[c] = m[c] = F2{0.0f, 0.0f};
        for (int q = lane; q < nc; q += 32) pair_contrib_f<true>(A, st, cb, k, q, f, m);
        if (lane < 6) wall_contrib_f<true>(A, st, k, lane, f, m);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                F2 of{__shfl_xor_sync(0xffffffffu, f[c].hi, off), __shfl_xor_sync(0xffffffffu, f[c].lo, off)};
                F2 om{__shfl_xor_sync(0xffffffffu, m[c].hi, off), __shfl_xor_sync(0xffffffffu, m[c].lo, off)};
                f[c] = f2_add(f[c], of);
                m[c] = f2_add(m[c], om);
            }
        if (lane == 0) {
            for (int a = 0; a < 3; ++a) {
                const double fa = (double)f[a].hi + (double)f[a].lo;
                const double ma = (double)m[a].hi + (double)m[a].lo;
                A.P.Fc[(long long)a * A.P.cap + k] = fa;
                A.P.Mc[(long long)a * A.P.cap + k] = ma;
                sF[w][a] = fa;
                sM[w][a] = ma;
            }
        }
    }
    if (!do_step) return;  // uniform across the CTA
    __syncthreads();
    const int kk = base + lane;
    if (w != 0 || lane >= wpc || kk >= A.P.n) return;
    double r[3], v[3], wv[3], d[9], Ft[3], Mt[3], acc[3];
    load_state(A, st, kk, r, v, wv, d);
    for (int a = 0; a < 3; ++a) {
        const long long o = (long long)a * A.P.cap + kk;
        Ft[a] = sF[lane][a] + A.P.Fhp[o];
        Mt[a] = sM[lane][a] + A.P.Mhp[o];
    }
    correct(A, kk, Ft, Mt, d, v, wv);
    for (int a = 0; a < 3; ++a) acc[a] = A.P.acc[(long long)a * A.P.cap + kk];
    predict(A, kk, r, v, acc, wv, d);
    store_state(A, A.P.st[out], kk, r, v, wv, d);
}

// Velocity update of the last substep (flowchart: after the fluid forces are reduced):
// corrector with the fresh hydrodynamic force (or none for DEM-only), result in buffer 0;
// the hydrodynamic force is held for the next step's substeps.
__global__ void k_final(DemArgs A, int in, int use_hydro) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.P.n) return;
    double r[3], v[3], w[3], d[9], F[3], M[3];
    load_state(A, A.P.st[in], k, r, v, w, d);
    for (int a = 0; a < 3; ++a) {
        long long o = (long long)a * A.P.cap + k;
        double fh = use_hydro ? A.P.Fh[o] : 0.0, mh = use_hydro ? A.P.Mh[o] : 0.0;
        F[a] = A.P.Fc[o] + fh;
        M[a] = A.P.Mc[o] + mh;
        A.P.Fhp[o] = fh;
        A.P.Mhp[o] = mh;
    }
    correct(A, k, F, M, d, v, w);
    bool bad = false;
    for (int a = 0; a < 3; ++a) bad |= !isfinite(v[a]) || !isfinite(w[a]);
    if (bad) atomicAdd(&A.status->nan_detected, 1);
    store_state(A, A.P.st[0], k, r, v, w, d);
}


// Contact forces of a substep, one warp per particle, from buffer `in` (Table 1 "Compute
// DEM forces" and "Reduce DEM forces"): stored in Fc, Mc.
__global__ void __launch_bounds__(128, 6) k_contacts(DemArgs A, int in, int cb) {
    const int k = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (k >= A.P.n) return;  // uniform across the warp
    double F[3], M[3];
    contact_sum_warp(A, A.P.st[in], cb, k, F, M);
    if ((threadIdx.x & 31) != 0) return;
    for (int a = 0; a < 3; ++a) {
        A.P.Fc[(long long)a * A.P.cap + k] = F[a];
        A.P.Mc[(long long)a * A.P.cap + k] = M[a];
    }
}



// ------------------------------------------------------------------------------------
// Batched DEM: one CTA per simulation runs the whole particle stage of a fluid step
// (candidate lists, every substep, the last contact sums) with CTA barriers between the
// phases instead of kernel launches. Candidates are found by direct search over the
// simulation's particles: for the small per-simulation counts this path serves it
// replaces the cell list and yields the same candidate lists (all particles within the
// sum of bounding radii plus the skin, ascending ids).
// ------------------------------------------------------------------------------------
__device__ void candidates_direct(const DemArgs& A, int i, int ob, int nbuf) {
    // one warp: lanes test ids base + lane, so ballot order is ascending id order
    const int lane = threadIdx.x & 31;
    const unsigned lower = (1u << lane) - 1u;
    const double* st = A.P.st[0];
    double ri[3];
    ld3(A, st, SP, i, ri);
    if (lane == 0)
        for (int a = 0; a < 3; ++a) A.P.pos_build[(long long)a * A.P.cap + i] = ri[a];
    const double bi = A.P.bound[i];
    int* nc = A.cand[nbuf] + (long long)i * A.ccap;
    int cnt = 0;
    for (int base = 0; base < A.P.n; base += 32) {
        const int j = base + lane;
        bool hit = false;
        if (j < A.P.n && j != i) {
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = min_image(A, a, ri[a] - stv(A, st, SP + a, j));
            double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double lim = bi + A.P.bound[j] + A.skin;
            hit = d2 < lim * lim;
        }
        const unsigned b = __ballot_sync(0xffffffffu, hit);
        const int pos = cnt + __popc(b & lower);
        if (hit && pos < A.ccap) nc[pos] = j;
        cnt += __popc(b);
    }
    if (cnt > A.ccap) {
        if (lane == 0) atomicAdd(&A.status->cand_overflow, 1);
        cnt = A.ccap;
    }
    __syncwarp();
    const int* oc = A.cand[ob] + (long long)i * A.ccap;
    const double* oh = A.hist[ob] + (long long)i * A.ccap * 3;
    double* nh = A.hist[nbuf] + (long long)i * A.ccap * 3;
    const int nold = A.ncand[ob][i];
    for (int m = lane; m < cnt; m += 32) {
        const int v = nc[m];
        int lo = 0, hi = nold;  // first old entry >= v
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (oc[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        const bool found = lo < nold && oc[lo] == v;
        for (int a = 0; a < 3; ++a) nh[3 * m + a] = found ? oh[3 * lo + a] : 0.0;
    }
    if (lane == 0) A.ncand[nbuf][i] = cnt;
}

__global__ void k_dem_batch(const DemArgs* args, const int* poff, int batch_parity) {
    const DemArgs& A = args[blockIdx.x];
    const int n = A.P.n;
    if (n == 0) return;  // uniform across the CTA
    const int p = batch_parity ^ poff[blockIdx.x];  // this member's buffer parity
    const int cb = p ^ 1, nsub = A.n_sub;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int k = warp; k < n; k += nwarps) candidates_direct(A, k, p, cb);
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double r[3], v[3], w[3], d[9], acc[3];
        load_state(A, A.P.st[0], k, r, v, w, d);
        for (int a = 0; a < 3; ++a) acc[a] = A.P.acc[(long long)a * A.P.cap + k];
        predict(A, k, r, v, acc, w, d);
        for (int a = 0; a < 3; ++a) A.P.st[0][(long long)(SP + a) * A.P.cap + k] = r[a];
        for (int m = 0; m < 9; ++m) A.P.st[0][(long long)(ST + m) * A.P.cap + k] = d[m];
    }
    __syncthreads();
    for (int sub = 1; sub <= nsub; ++sub) {
        const int in = (sub - 1) & 1, out = sub & 1;
        for (int k = warp; k < n; k += nwarps) {
            double F[3], M[3];
            contact_sum_warp(A, A.P.st[in], cb, k, F, M);
            if (lane == 0)
                for (int a = 0; a < 3; ++a) {
                    A.P.Fc[(long long)a * A.P.cap + k] = F[a];
                    A.P.Mc[(long long)a * A.P.cap + k] = M[a];
                }
        }
        __syncthreads();
        if (sub == nsub) break;  // the last substep's velocities wait for the fluid
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            double r[3], v[3], w[3], d[9], Ft[3], Mt[3], acc[3];
            load_state(A, A.P.st[in], k, r, v, w, d);
            for (int a = 0; a < 3; ++a) {
                long long o = (long long)a * A.P.cap + k;
                Ft[a] = A.P.Fc[o] + A.P.Fhp[o];
                Mt[a] = A.P.Mc[o] + A.P.Mhp[o];
            }
            correct(A, k, Ft, Mt, d, v, w);
            for (int a = 0; a < 3; ++a) acc[a] = A.P.acc[(long long)a * A.P.cap + k];
            predict(A, k, r, v, acc, w, d);
            store_state(A, A.P.st[out], k, r, v, w, d);
        }
        __syncthreads();
    }
}

__global__ void k_final_batch(const DemArgs* args, int use_hydro_mask) {
    const DemArgs& A = args[blockIdx.x];
    const int n = A.P.n;
    const int in = (A.n_sub - 1) & 1;
    const int use_hydro = (use_hydro_mask >> 0) & 1;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double r[3], v[3], w[3], d[9], F[3], M[3];
        load_state(A, A.P.st[in], k, r, v, w, d);
        for (int a = 0; a < 3; ++a) {
            long long o = (long long)a * A.P.cap + k;
            double fh = use_hydro ? A.P.Fh[o] : 0.0, mh = use_hydro ? A.P.Mh[o] : 0.0;
            F[a] = A.P.Fc[o] + fh;
            M[a] = A.P.Mc[o] + mh;
            A.P.Fhp[o] = fh;
            A.P.Mhp[o] = mh;
        }
        correct(A, k, F, M, d, v, w);
        bool bad = false;
        for (int a = 0; a < 3; ++a) bad |= !isfinite(v[a]) || !isfinite(w[a]);
        if (bad) atomicAdd(&A.status->nan_detected, 1);
        store_state(A, A.P.st[0], k, r, v, w, d);
    }
}

cudaError_t launch_dem_batch(const DemArgs* args, const int* poff, int nsim, int p, cudaStream_t s) {
    k_dem_batch<<<nsim, 256, 0, s>>>(args, poff, p);
    return cudaGetLastError();
}

cudaError_t launch_final_batch(const DemArgs* args, int nsim, cudaStream_t s) {
    k_final_batch<<<nsim, 128, 0, s>>>(args, 1);
    return cudaGetLastError();
}

// Contact set at buffer 0 positions: counts of partners j > i, then keys (i << 32 | j).
__global__ void k_pair_count(DemArgs A, int cb, uint32_t* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.P.n) return;
    const int nc = A.ncand[cb][i];
    const int* cl = A.cand[cb] + (long long)i * A.ccap;
    uint32_t c = 0;
    for (int m = 0; m < nc; ++m) {
        int j = cl[m];
        if (j <= i) continue;
        Geo g;
        c += pair_geo(A, A.P.st[0], i, j, g) ? 1u : 0u;
    }
    cnt[i] = c;
}

__global__ void k_pair_emit(DemArgs A, int cb, const uint32_t* off, unsigned long long* keys, int cap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.P.n) return;
    const int nc = A.ncand[cb][i];
    const int* cl = A.cand[cb] + (long long)i * A.ccap;
    uint32_t o = off[i];
    for (int m = 0; m < nc; ++m) {
        int j = cl[m];
        if (j <= i) continue;
        Geo g;
        if (pair_geo(A, A.P.st[0], i, j, g)) {
            if ((int)o < cap) keys[o] = ((unsigned long long)i << 32) | (unsigned)j;
            ++o;
        }
    }
}

// ------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------
static inline unsigned nblk(int n, int t) { return (unsigned)((n + t - 1) / t); }

// Neighbour rebuild from the positions of state buffer pst: cell keys, counting sort,
// candidate lists (old buffer ob -> new buffer nb, histories carried over).
cudaError_t launch_rebuild(const DemArgs& A, int ob, int nb, int pst, uint32_t* scan_partial, cudaStream_t s,
                           int* launches) {
    int n = A.P.n;
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(A.cell_count, 0, sizeof(uint32_t) * (A.G + 1), s);
    if (e != cudaSuccess) return e;
    k_keys<<<nblk(n, 128), 128, 0, s>>>(A, pst);
    e = launch_scan(A.cell_count, A.G, A.cell_start, scan_partial, s);
    if (e != cudaSuccess) return e;
    k_scatter<<<nblk(n, 128), 128, 0, s>>>(A);
    e = launch_segsort(A.cell_start, A.G, n, A.sorted_tmp, A.sorted, A.seg_big, s);
    if (e != cudaSuccess) return e;
    k_candidates<<<nblk(n, CAND_WARPS), 32 * CAND_WARPS, 0, s>>>(A, ob, nb, pst);
    *launches += 8;
    if (A.pair_once) {  // canonical pair list of the new candidate lists
        k_cpair_count<<<nblk(n, 128), 128, 0, s>>>(A, nb, A.cp_cnt);
        e = launch_scan(A.cp_cnt, n, A.cp_off, scan_partial, s);
        if (e != cudaSuccess) return e;
        k_cpair_emit<<<nblk(n, 128), 128, 0, s>>>(A, nb, A.cp_off, A.cp_list);
        *launches += 5;
    }
    return cudaGetLastError();
}

cudaError_t launch_predict_first(const DemArgs& A, cudaStream_t s) {
    if (A.P.n <= 0) return cudaSuccess;
    k_predict_first<<<nblk(A.P.n, 128), 128, 0, s>>>(A);
    return cudaGetLastError();
}

// do_step = 1: contact forces then corrector + next predictor (in -> out);
// do_step = 0: contact forces only.
cudaError_t launch_substep(const DemArgs& A, int in, int out, int cb, int do_step, int* launches, cudaStream_t s) {
    if (A.P.n <= 0) return cudaSuccess;
    if (!A.pair_once && A.force_f32) {  // spheres only, FP32 contacts: one launch per substep
        // particles per CTA: spread over every SM (the contact arithmetic loads the SM's FP64
        // pipe in proportion to its particles), at most SUB_WARPS
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int wpc = std::min(SUB_WARPS, std::max(1, (A.P.n + nsm - 1) / std::max(nsm, 1)));
        k_substep_spheres<<<nblk(A.P.n, wpc), 32 * wpc, 0, s>>>(A, in, out, cb, do_step);
        *launches += 1;
        return cudaGetLastError();
    }
    *launches += (A.pair_once ? 2 : 1) + (do_step ? 1 : 0);
    if (A.pair_once) {
        const long long maxp = (long long)A.P.n * A.ccap;  // every slot may hold an owned pair
        k_pair_forces<<<(unsigned)((maxp + 127) / 128), 128, 0, s>>>(A, in, cb, A.cp_off, A.cp_list, A.cp_res,
                                                                     A.cp_stride);
        k_contacts_gather<<<nblk(A.P.n * 32, 128), 128, 0, s>>>(A, in, cb, A.cp_off, A.cp_res, A.cp_stride);
    } else {
        k_contacts<<<nblk(A.P.n * 32, 128), 128, 0, s>>>(A, in, cb);
    }
    if (do_step) k_integrate<<<nblk(A.P.n, 32), 32, 0, s>>>(A, in, out);
    return cudaGetLastError();
}

cudaError_t launch_final(const DemArgs& A, int in, int use_hydro, cudaStream_t s) {
    if (A.P.n <= 0) return cudaSuccess;
    k_final<<<nblk(A.P.n, 128), 128, 0, s>>>(A, in, use_hydro);
    return cudaGetLastError();
}

cudaError_t launch_pairs(const DemArgs& A, int cb, uint32_t* cnt, uint32_t* off, uint32_t* partial,
                         unsigned long long* keys, int cap, cudaStream_t s) {
    if (A.P.n <= 0) return cudaSuccess;
    k_pair_count<<<nblk(A.P.n, 64), 64, 0, s>>>(A, cb, cnt);
    cudaError_t e = launch_scan(cnt, A.P.n, off, partial, s);
    if (e != cudaSuccess) return e;
    k_pair_emit<<<nblk(A.P.n, 64), 64, 0, s>>>(A, cb, off, keys, cap);
    return cudaGetLastError();
}

}  // namespace ledds
