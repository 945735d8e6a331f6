// Template instantiations of the OCI / SI kernels for R = float.
#include <cstdlib>

#include "oci_kernels.h"

namespace ocik {

constexpr int kStages = 2;

template <int LPC, int PPL, int CHUNK>
static void fill(KernelSet *k)
{
    k->cells_oci = (const void *)&k_cells<float, LPC, PPL, CHUNK, M_OCI>;
    k->cells_si = (const void *)&k_cells<float, LPC, PPL, CHUNK, M_SI>;
    k->commit_oci = (const void *)&k_percell<float, LPC, PPL, C_COMMIT_OCI>;
    k->commit_si = (const void *)&k_percell<float, LPC, PPL, C_COMMIT_SI>;
    k->si_prep = (const void *)&k_percell<float, LPC, PPL, C_SI_PREP>;
    k->guess = (const void *)&k_percell<float, LPC, PPL, C_GUESS>;
    k->march = (const void *)&k_si_march<float>;
    k->scan_reduce = (const void *)&k_scan_reduce<float>;
    k->scan_segments = (const void *)&k_scan_segments<float>;
    k->scan_apply = (const void *)&k_scan_apply<float>;
    k->be_cells = (const void *)&k_be_cells<float>;
    k->be_commit = (const void *)&k_be_commit<float>;
    k->lift_guess = (const void *)&k_lift<float, LPC, PPL, LIFT_GUESS>;
    k->lift_corr = (const void *)&k_lift<float, LPC, PPL, LIFT_CORR>;
    k->cells_oci_tma = nullptr;
    k->cells_oci_loop = nullptr;
    k->cells_si_tma = nullptr;
    k->cells_lin_tma = nullptr;
    k->tma_stages = 0;
    if constexpr (LPC >= 2) {
        k->cells_oci_tma = (const void *)&k_cells_tma<LPC, PPL, CHUNK, kStages, M_OCI>;
        k->cells_oci_loop = (const void *)&k_cells_tma<LPC, PPL, CHUNK, kStages, M_OCI, true>;
        k->cells_si_tma = (const void *)&k_cells_tma<LPC, PPL, CHUNK, kStages, M_SI>;
        k->cells_lin_tma = (const void *)&k_cells_tma<LPC, PPL, CHUNK, kStages, M_LIN>;
        k->tma_stages = kStages;
        k->tma_chunk = CHUNK;
        k->tma_max_warps = tma_max_threads(CHUNK, PPL) / 32;
    }
    k->commit_lin = (const void *)&k_percell<float, LPC, PPL, C_COMMIT_LIN>;
    k->refine = (const void *)&k_refine_residual<LPC, PPL>;
    k->cells_per_warp = CHUNK * (32 / LPC);
    k->cells_per_warp_pc = 32 / LPC;
}

bool kernel_set_f32(int lpc, int ppl, KernelSet *out)
{
    switch (lpc * 16 + ppl) {
    case 1 * 16 + 1: fill<1, 1, 8>(out); return true;
    case 2 * 16 + 1: fill<2, 1, 8>(out); return true;
    case 4 * 16 + 1: fill<4, 1, 8>(out); return true;
    case 8 * 16 + 1: fill<8, 1, 8>(out); return true;
    case 16 * 16 + 1: fill<16, 1, 8>(out); return true;
    case 32 * 16 + 1:
        fill<32, 1, 8>(out);
        if (const char *e = std::getenv("OCI_TMA_STAGES"); e && e[0] == '3') {
            out->cells_oci_tma = (const void *)&k_cells_tma<32, 1, 8, 3, M_OCI>;
            out->cells_oci_loop = (const void *)&k_cells_tma<32, 1, 8, 3, M_OCI, true>;
            out->cells_si_tma = (const void *)&k_cells_tma<32, 1, 8, 3, M_SI>;
            out->cells_lin_tma = (const void *)&k_cells_tma<32, 1, 8, 3, M_LIN>;
            out->tma_stages = 3;
        }
        return true;
    case 32 * 16 + 2: fill<32, 2, 8>(out); return true;
    case 32 * 16 + 4: fill<32, 4, 4>(out); return true;
    default: return false;
    }
}

unsigned tma_stage_bytes(int lpc, int chunk, int P)
{
    const unsigned cpc = (unsigned)(chunk * (32 / lpc));
    return round16(cpc * P * 8u) * 2u + round16(cpc * P * 16u) + round16(cpc * 16u) + round16(cpc * 4u);
}

}  // namespace ocik
