// psm_wide.cu -- the PSM kernel for lattices whose populations need 64-bit element
// offsets (19 N >= 2^31 elements, e.g. more than 1.1e8 cells), in each step form: the
// two-lattice pull and the two steps of the AA pattern. The arithmetic is that of the
// 32-bit-offset kernels; only the plane offsets i N and the pulled indices are 64-bit.
#include "internal.cuh"
#include "psm.cuh"

namespace ledds {

cudaError_t launch_psm_wide(const LbmArgs& a, const PsmMaps* m, int store, cudaStream_t s) {
    if (a.aa == PSM_AB) return launch_psm_mode<PSM_AB | PSM_W64>(a, m, store, s);
    if (a.pop_in != a.pop_out) return cudaErrorInvalidValue;
    if (a.aa == PSM_AA_EVEN) return launch_psm_mode<PSM_AA_EVEN | PSM_W64>(a, m, store, s);
    if (a.aa == PSM_AA_ODD) return launch_psm_mode<PSM_AA_ODD | PSM_W64>(a, m, store, s);
    return cudaErrorInvalidValue;
}

}  // namespace ledds
