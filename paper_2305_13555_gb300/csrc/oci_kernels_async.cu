// Template instantiations of the barrier-free persistent OCI loop
// (k_cells_tma ASYNC) for the layouts of S_32, S_64 and S_128.  A translation
// unit of its own so the build compiles it beside the FP32 set.
#include "oci_kernels.h"

namespace ocik {

const void *kernel_async_loop(int lpc, int ppl)
{
    switch (lpc * 16 + ppl) {
    case 16 * 16 + 1: return (const void *)&k_cells_tma<16, 1, 8, 2, M_OCI, true, 0, true>;
    case 32 * 16 + 1: return (const void *)&k_cells_tma<32, 1, 8, 2, M_OCI, true, 0, true>;
    case 32 * 16 + 2: return (const void *)&k_cells_tma<32, 2, 8, 2, M_OCI, true, 0, true>;
    default: return nullptr;
    }
}

}  // namespace ocik
