// psm_aa.cu -- the PSM kernel on a single population array (the AA pattern): the two
// step forms alternate, an in-place collision that leaves f*_i in slot opp(i) of its own
// node, then a step that reads f*_i(x - c_i) from there, collides, and pushes f*_i(x)
// to slot i of x + c_i (or back to x at a wall). Every array slot is then read and
// written by one node only, so the step needs no second array and no synchronisation
// beyond the kernel boundary; the arithmetic per node is that of the two-lattice pull.
#include "internal.cuh"
#include "psm.cuh"

namespace ledds {

cudaError_t launch_psm_aa(const LbmArgs& a, const PsmMaps* m, int store, cudaStream_t s) {
    if (a.pop_in != a.pop_out) return cudaErrorInvalidValue;
    if (a.aa == PSM_AA_EVEN) return launch_psm_mode<PSM_AA_EVEN>(a, m, store, s);
    if (a.aa == PSM_AA_ODD) return launch_psm_mode<PSM_AA_ODD>(a, m, store, s);
    return cudaErrorInvalidValue;
}

}  // namespace ledds
