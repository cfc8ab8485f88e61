// psm_aa.cu -- the PSM kernel on a single population array (the AA pattern): the two
// step forms alternate, an in-place collision that leaves f*_i in slot opp(i) of its own
// node, then a step that reads f*_i(x - c_i) from there, collides, and pushes f*_i(x)
// to slot i of x + c_i (or back to x at a wall). Every array slot is then read and
// written by one node only, so the step needs no second array and no synchronisation
// beyond the kernel boundary; the arithmetic per node is that of the two-lattice pull.
#include "internal.cuh"
#include "psm.cuh"

namespace ledds {

template <int STORE, bool TRT, int MODE>
static cudaError_t launch_aa_t(const LbmArgs& a, cudaStream_t s) {
    static bool configured = false;
    const size_t smem = psm_smem_bytes(STORE);
    if (!configured) {
        cudaError_t e =
            cudaFuncSetAttribute(k_psm<STORE, TRT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_psm<STORE, TRT, MODE><<<dim3(a.ntx, a.nty, a.ntz * a.zsplit), PSM_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_aa_mode(const LbmArgs& a, int store, cudaStream_t s) {
    if (a.trt) {
        if (store == LEDDS_STORE_F32) return launch_aa_t<LEDDS_STORE_F32, true, MODE>(a, s);
        if (store == LEDDS_STORE_F16) return launch_aa_t<LEDDS_STORE_F16, true, MODE>(a, s);
        return launch_aa_t<LEDDS_STORE_BF16, true, MODE>(a, s);
    }
    if (store == LEDDS_STORE_F32) return launch_aa_t<LEDDS_STORE_F32, false, MODE>(a, s);
    if (store == LEDDS_STORE_F16) return launch_aa_t<LEDDS_STORE_F16, false, MODE>(a, s);
    return launch_aa_t<LEDDS_STORE_BF16, false, MODE>(a, s);
}

cudaError_t launch_psm_aa(const LbmArgs& a, int store, cudaStream_t s) {
    if (a.pop_in != a.pop_out) return cudaErrorInvalidValue;
    if (a.aa == PSM_AA_EVEN) return launch_aa_mode<PSM_AA_EVEN>(a, store, s);
    if (a.aa == PSM_AA_ODD) return launch_aa_mode<PSM_AA_ODD>(a, store, s);
    return cudaErrorInvalidValue;
}

}  // namespace ledds
