// Template instantiations of the staged FP32 OCI iteration with BF16 face
// storage, for the layouts of S_32 (16 lanes per cell), S_64 (32 lanes) and
// S_128 (32 lanes, two pairs per lane).  A translation unit of its own so the
// build compiles it beside the FP32 set.
#include "oci_kernels.h"

namespace ocik {

constexpr int kStagesH = 2;

template <int LPC, int PPL, int CHUNK>
static void fill_halo(HaloKernels *k)
{
    k->entry = (const void *)&k_cells_tma<LPC, PPL, CHUNK, kStagesH, M_OCI, false, 1>;
    k->loop = (const void *)&k_cells_tma<LPC, PPL, CHUNK, kStagesH, M_OCI, true, 2>;
    k->exit = (const void *)&k_cells_tma<LPC, PPL, CHUNK, kStagesH, M_OCI, false, 3>;
}

bool kernel_set_bf16(int lpc, int ppl, HaloKernels *out)
{
    switch (lpc * 16 + ppl) {
    case 16 * 16 + 1: fill_halo<16, 1, 8>(out); return true;
    case 32 * 16 + 1: fill_halo<32, 1, 8>(out); return true;
    case 32 * 16 + 2: fill_halo<32, 2, 8>(out); return true;
    default: return false;
    }
}

}  // namespace ocik
