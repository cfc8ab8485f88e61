// internal.cuh -- shared device definitions of the LEDDS GB300 library.
//
// D3Q19 lattice tables (Sec. 2.3), storage formats of the populations, kernel argument
// structs and the launch helpers used by lbm.cu, dem.cu and api.cu.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ledds.h"

namespace ledds {

// ------------------------------------------------------------------------------------
// D3Q19 velocity set in the order documented in ledds.h: rest; +x,-x,+y,-y,+z,-z; then
// the 12 edge velocities, each followed by its opposite. Written as constexpr functions
// so that fully unrolled loops fold every table entry into an immediate.
// ------------------------------------------------------------------------------------
__host__ __device__ constexpr int CX(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)   ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int CY(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)   ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18)  ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int CZ(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)  ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                   : 0;
}
__host__ __device__ constexpr float TW(int i) {
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr int OPP(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// ------------------------------------------------------------------------------------
// Population storage: g_i = f_i - t_i in FP32, FP16 or BF16; 16-bit formats keep
// g_i * 2^s (s = storage_scale_log2) to stay clear of FP16 subnormals.
// ------------------------------------------------------------------------------------
template <int STORE>
struct Store;

template <>
struct Store<LEDDS_STORE_F32> {
    using T = float;
    static __device__ __forceinline__ float load(const T* p, float) { return *p; }
    // stored units (the PSM kernel works on stored values and scales its moments)
    static __device__ __forceinline__ float raw(T v) { return v; }
    static __device__ __forceinline__ float ldg_raw(const T* p) { return __ldg(p); }
    static __device__ __forceinline__ void store_raw(T* p, float v) { __stcs(p, v); }
    // streaming store under a predicate (no branch around it)
    static __device__ __forceinline__ void store_if(T* p, float v, bool pred) {
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.cs.f32 [%0], %1;\n\t}" ::"l"(p),
                     "f"(v), "r"((unsigned)pred)
                     : "memory");
    }
    static __device__ __forceinline__ float up(float v, float) { return v; }
    static __device__ __forceinline__ float from_bits(unsigned short, float) { return 0.f; }
    static __device__ __forceinline__ void store(T* p, float v, float) { __stcs(p, v); }
};
template <>
struct Store<LEDDS_STORE_F16> {
    using T = __half;
    static __device__ __forceinline__ float load(const T* p, float inv) {
        return __half2float(*p) * inv;
    }
    static __device__ __forceinline__ float raw(T v) { return __half2float(v); }
    static __device__ __forceinline__ float ldg_raw(const T* p) {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
    }
    static __device__ __forceinline__ void store_raw(T* p, float v) {
        __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(__float2half_rn(v)));
    }
    static __device__ __forceinline__ void store_if(T* p, float v, bool pred) {
        const unsigned short h = __half_as_ushort(__float2half_rn(v));
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.cs.b16 [%0], %1;\n\t}" ::"l"(p),
                     "h"(h), "r"((unsigned)pred)
                     : "memory");
    }
    static __device__ __forceinline__ float up(float v, float scale) { return v * scale; }
    static __device__ __forceinline__ float from_bits(unsigned short h, float inv) {
        return __half2float(__ushort_as_half(h)) * inv;
    }
    static __device__ __forceinline__ void store(T* p, float v, float scale) {
        __stcs(reinterpret_cast<unsigned short*>(p),
               __half_as_ushort(__float2half_rn(v * scale)));
    }
};
template <>
struct Store<LEDDS_STORE_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float load(const T* p, float inv) {
        return __bfloat162float(*p) * inv;
    }
    static __device__ __forceinline__ float raw(T v) { return __bfloat162float(v); }
    static __device__ __forceinline__ float ldg_raw(const T* p) {
        return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p))));
    }
    static __device__ __forceinline__ void store_raw(T* p, float v) {
        __stcs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(__float2bfloat16_rn(v)));
    }
    static __device__ __forceinline__ void store_if(T* p, float v, bool pred) {
        const unsigned short h = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.cs.b16 [%0], %1;\n\t}" ::"l"(p),
                     "h"(h), "r"((unsigned)pred)
                     : "memory");
    }
    static __device__ __forceinline__ float up(float v, float scale) { return v * scale; }
    static __device__ __forceinline__ float from_bits(unsigned short h, float inv) {
        return __bfloat162float(__ushort_as_bfloat16(h)) * inv;
    }
    static __device__ __forceinline__ void store(T* p, float v, float scale) {
        __stcs(reinterpret_cast<unsigned short*>(p),
               __bfloat16_as_ushort(__float2bfloat16_rn(v * scale)));
    }
};

inline size_t storage_bytes(int store) { return store == LEDDS_STORE_F32 ? 4 : 2; }
__host__ __device__ constexpr int storage_bytes_c(int store) { return store == LEDDS_STORE_F32 ? 4 : 2; }

// Lattice tile handled by one CTA of the PSM kernel: 32 x 8 nodes per plane (one warp
// per x-row), TILE_Z planes.
constexpr int TILE_X = 32;
constexpr int TILE_Y = 8;
constexpr int TILE_Z = 16;       // tile depth of a simulation (a batch may choose another)
constexpr int TILE_Z_MIN = 8;    // smallest tile depth; tile lists are sized for it
constexpr int MAX_TILE_CAP = 64;
constexpr int MAX_CAND_CAP = 64;

// Device status counters (one struct in the workspace).
struct DevStatus {
    unsigned long long steps;
    int tile_overflow;
    int cand_overflow;
    int solids_overflow;
    int skin_violation;
    int ell_nonconverged;
    int nan_detected;
    int wait_timeout;             // bounded waits of the staged PSM pipeline that gave up
    int pad;
};

// Particle arrays in the workspace. State buffers hold [18][cap] doubles: pos xyz,
// vel xyz, omega xyz, triad d1 d2 d3.
struct DevParticles {
    int n, cap;
    double* st[2];
    double *acc, *alpha;          // [3][cap]
    double *Fc, *Mc;              // contact force/torque of the last substep
    double *Fh, *Mh;              // hydrodynamic force/torque of the last fluid step
    double *Fhp, *Mhp;            // held hydrodynamic force/torque for substeps
    double* pos_build;            // positions at the last neighbour rebuild
    double *radius, *semi, *bound, *mass, *inertia, *gfac;  // semi, inertia: [3][cap]
    int* shape;
};

// Population array patterns, which are also the PSM kernel's step forms: the two-lattice
// pull (AB), and the in-place AA pattern's two alternating steps. A kernel's MODE is the
// form, plus PSM_W64 when the populations need 64-bit element offsets (19 N >= 2^31).
enum { PSM_AB = 0, PSM_AA_EVEN = 1, PSM_AA_ODD = 2, PSM_W64 = 4 };
__host__ __device__ constexpr int psm_form(int mode) { return mode & 3; }
__host__ __device__ constexpr bool psm_w64(int mode) { return (mode & PSM_W64) != 0; }

// Offsets of the state buffer components.
constexpr int SP = 0, SV = 3, SW = 6, ST = 9;

struct LbmArgs {
    int nx, ny, nz;
    long long N;
    int per[3];
    float uw[3][2][3];
    float tau, omega;
    float F[3];
    int has_force;
    float guo_pref;               // 1 - 1/(2 tau)
    int trt;                      // TRT collision: odd parts relax at omega_m
    float omega_m, guo_pref_m;    // 1/tau- and 1 - 1/(2 tau-)
    float scale, inv_scale;
    const void* pop_in;
    void* pop_out;                // the same array as pop_in with the AA pattern
    int pN[19];                   // i * N: start of plane i (19 N < 2^31 is required)
    int off[19];                  // c_x + nx c_y + nx ny c_z: pull offset of direction i
    unsigned off_odd;             // bit i: off[i] is odd (16-bit word selection)
    int nx_even;                  // nx even: a pulled index has the parity of x - c_x
    int mi[3];                    // per axis: node-particle offsets may need a periodic wrap
    // tile lists (tiles of TILE_X x TILE_Y x tz nodes)
    int ntx, nty, ntz, tile_cap;
    int tz;
    int zsplit;                   // CTAs per tile of the PSM kernel (1, or more for small lattices)
    const int* tile_count;
    const int* tile_ids;
    // particles (the state buffer the fluid step sees)
    const double* st;
    int pcap;
    const double *radius, *semi, *bound;
    const int* shape;
    double *Fh, *Mh;
    int voxel, subdiv_n;
    int subdiv_any;               // subdivision fractions requested or some particle an ellipsoid
    float Rc, inv2Rc;
    DevStatus* status;
    // (last: the PSM kernel is measurably faster with pN at the 16-byte-aligned offset it
    // has without this field in front of it)
    int aa;                       // pattern of the array: PSM_AB (two lattices), or one array
                                  // (AA) holding PSM_AA_EVEN: pre-collision f, natural slots,
                                  // or PSM_AA_ODD: post-collision f*_i in slot opp(i)
    int w64;                      // 64-bit plane offsets (pN unused): 19 N >= 2^31 or requested
};

// Arguments of one batched PSM launch: up to BATCH_CHUNK members and the prefix sums of
// their tile counts (passed by value: 64 x 488 bytes fit the 32 KB parameter limit).
constexpr int BATCH_CHUNK = 64;
struct BatchChunk {
    LbmArgs a[BATCH_CHUNK];
    int tile_start[BATCH_CHUNK + 1];
    int nsim;
};
static_assert(sizeof(BatchChunk) <= 32764, "a batch chunk must fit the kernel parameter space");

// Tensor maps of one population array for the staged PSM route (4D: x, y, z, plane; boxes
// of TILE_Y rows by TILE_X or TILE_X + 2H columns, one plane deep), made by psm_make_maps.
struct PsmMaps {
    CUtensorMap narrow, wide;
};
bool psm_make_maps(const void* pop, int store, int nx, int ny, int nz, PsmMaps* out);  // lbm.cu

struct DemArgs {
    DevParticles P;
    // domain
    double lo[3], hi[3], L[3];
    int per[3];
    double uw[3][2][3];
    // grid
    int gn[3];
    double gh[3];
    int G;
    // parameters
    double dt;
    int n_sub;
    double gravity[3];
    int law;
    double k_n, k_t, beta, Ystar, Gstar, mu;
    double skin;
    int ell_max_iter;
    double ell_tol;
    int ell_screen;   // exact disjointness screens before the ellipsoid iteration
    int force_f32;  // FP32 contact arithmetic, FP64 sums
    int quat;       // quaternion orientation update in the predictor
    // pair-once evaluation (simulations with ellipsoids): canonical pair counts, offsets
    // (n + 1), list (i * MAX_CAND_CAP + slot) and results [9][cp_stride]
    int pair_once;
    uint32_t *cp_cnt, *cp_off, *cp_list;
    void* cp_res;
    long long cp_stride;
    // lists
    int ccap;
    uint32_t* keys;
    int* rank;
    int* sorted;
    int* sorted_tmp;              // ids in scatter order (before each cell is ordered)
    int* seg_big;                 // cells of more than SEG_SMALL ids: count, list
    uint32_t* cell_count;
    uint32_t* cell_start;
    int* cand[2];
    int* ncand[2];
    double* hist[2];
    double* whist;
    DevStatus* status;
};

}  // namespace ledds
