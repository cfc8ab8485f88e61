// noalloc.cu -- the DEM cell list (keys and (key, id)-sorted ids) computed without any
// device allocation, for callers that cannot allocate device memory themselves (see
// ledds_cell_list_noalloc in include/ledds.h).
//
// The scratch the counting sort needs (per-cell counts and starts, scan partials,
// per-particle ranks, the ids in scatter order and the list of large cells) lives in one
// file-scope __device__ array of fixed size (about 4.2 MB). Every GPU that loads the
// library holds it until the process exits. Host code cannot use the array's name as a
// device address: the address is looked up once per CUDA context with
// cudaGetSymbolAddress and passed to the kernels.
#include <cudaTypedefs.h>
#include <math.h>

#include <mutex>

#include "internal.cuh"

namespace ledds {
cudaError_t launch_scan(const uint32_t* in, int n, uint32_t* out, uint32_t* partial, cudaStream_t s);
cudaError_t launch_segsort(const uint32_t* start, int G, int n, const int* tmp, int* sorted, int* big,
                           cudaStream_t s);
}
using namespace ledds;

namespace {

constexpr int kMaxCells = 1 << 18;      // grid cells
constexpr int kMaxParticles = 1 << 18;  // particles
constexpr int kPartials = 4096;         // scan block partials
// counts [cells+1] | starts [cells+1] | partials [4096] | ranks [particles] |
// ids in scatter order [particles] | large-cell list [particles/32 + 2]
constexpr size_t kWords = 2 * ((size_t)kMaxCells + 1) + kPartials + 2 * (size_t)kMaxParticles +
                          kMaxParticles / 32 + 2;

__device__ __align__(256) uint32_t g_scratch[kWords];

// The scratch address per CUDA context: a context (and the library's module in it) can be
// destroyed and made again on the same device (cudaDeviceReset, or the primary context
// released and retained), and the array then has a new address.
constexpr int kSlots = 64;
std::mutex g_mu;
CUcontext g_ctx[kSlots] = {nullptr};
uint32_t* g_addr[kSlots] = {nullptr};
PFN_cuCtxGetCurrent_v4000 g_get_ctx = nullptr;

// Device address of the scratch array in the current context.
int scratch_address(uint32_t** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_get_ctx) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return LEDDS_ERR_CUDA;
        g_get_ctx = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    }
    CUcontext ctx = nullptr;
    void* p = nullptr;
    if (g_get_ctx(&ctx) != CUDA_SUCCESS) return LEDDS_ERR_CUDA;
    if (!ctx) {
        // no context is current yet: the symbol lookup makes the device's primary one current
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return LEDDS_ERR_CUDA;
        if (g_get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return LEDDS_ERR_CUDA;
    }
    int slot = -1;
    for (int i = 0; i < kSlots && slot < 0; ++i)
        if (g_ctx[i] == ctx) slot = i;
    if (slot < 0 || !g_addr[slot]) {
        if (!p && (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p)) return LEDDS_ERR_CUDA;
        if (slot < 0) {
            for (int i = 0; i < kSlots && slot < 0; ++i)
                if (!g_ctx[i]) slot = i;
            if (slot < 0) slot = (int)(reinterpret_cast<uintptr_t>(ctx) % kSlots);  // table full: reuse
        }
        g_ctx[slot] = ctx;
        g_addr[slot] = static_cast<uint32_t*>(p);
    }
    *out = g_addr[slot];
    return LEDDS_OK;
}

struct Grid {
    double lo[3], gh[3];
    int gn[3];
};

// key = k_x + n_x (k_y + n_y k_z), k_a = floor((r_a - lo_a)/h_a) clamped to [0, n_a - 1]
__global__ void k_na_keys(const double* pos, int n, Grid g, uint32_t* keys, uint32_t* count,
                          uint32_t* rank) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int c[3];
    for (int a = 0; a < 3; ++a) {
        double q = floor((pos[(long long)a * n + k] - g.lo[a]) / g.gh[a]);
        // clamp before converting: a non-finite position lands in cell 0, never out of range
        int v;
        if (!(q >= 0.0)) v = 0;
        else if (q > g.gn[a] - 1) v = g.gn[a] - 1;
        else v = (int)q;
        c[a] = v;
    }
    uint32_t key = (uint32_t)(c[0] + g.gn[0] * (c[1] + g.gn[1] * c[2]));
    keys[k] = key;
    rank[k] = atomicAdd(&count[key], 1u);
}

__global__ void k_na_scatter(const uint32_t* keys, const uint32_t* rank, const uint32_t* start, int n,
                             int* sorted) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    sorted[start[keys[k]] + rank[k]] = k;
}

}  // namespace

extern "C" int ledds_cell_list_noalloc(const double* d_pos, int n, const double box_lo[3],
                                       const double box_hi[3], double h, uint32_t* d_keys,
                                       int32_t* d_sorted_ids, int grid_n[3], void* stream) {
    if (!box_lo || !box_hi || !(h > 0.0) || n < 0) return LEDDS_ERR_INVALID_ARG;
    if (n > 0 && (!d_pos || !d_keys || !d_sorted_ids)) return LEDDS_ERR_INVALID_ARG;
    Grid g;
    long long G = 1;
    for (int a = 0; a < 3; ++a) {
        double L = box_hi[a] - box_lo[a];
        if (!(L > 0.0)) return LEDDS_ERR_INVALID_ARG;
        double q = floor(L / h);
        int c = q < 1.0 ? 1 : (q > (double)kMaxCells ? kMaxCells + 1 : (int)q);
        g.lo[a] = box_lo[a];
        g.gn[a] = c;
        g.gh[a] = L / c;
        G *= c;
    }
    if (grid_n)
        for (int a = 0; a < 3; ++a) grid_n[a] = g.gn[a];
    if (G > kMaxCells || n > kMaxParticles) return LEDDS_ERR_CAPACITY;
    if (n == 0) return LEDDS_OK;
    uint32_t* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != LEDDS_OK) return rc;
    uint32_t* count = base;
    uint32_t* start = count + (kMaxCells + 1);
    uint32_t* partial = start + (kMaxCells + 1);
    uint32_t* rank = partial + kPartials;
    int* tmp = reinterpret_cast<int*>(rank + kMaxParticles);
    int* big = tmp + kMaxParticles;
    cudaStream_t s = (cudaStream_t)stream;
    // the scratch keeps the previous call's contents: the counts (and the large-cell
    // counter, cleared by launch_segsort) must start at zero
    if (cudaMemsetAsync(count, 0, sizeof(uint32_t) * (size_t)(G + 1), s) != cudaSuccess) return LEDDS_ERR_CUDA;
    k_na_keys<<<(n + 127) / 128, 128, 0, s>>>(d_pos, n, g, d_keys, count, rank);
    if (launch_scan(count, (int)G, start, partial, s) != cudaSuccess) return LEDDS_ERR_CUDA;
    k_na_scatter<<<(n + 127) / 128, 128, 0, s>>>(d_keys, rank, start, n, tmp);
    if (launch_segsort(start, (int)G, n, tmp, d_sorted_ids, big, s) != cudaSuccess) return LEDDS_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? LEDDS_OK : LEDDS_ERR_CUDA;
}
