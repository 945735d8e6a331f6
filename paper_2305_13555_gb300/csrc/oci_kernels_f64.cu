// Template instantiations of the OCI / SI kernels for R = double.
#include "oci_kernels.h"

namespace ocik {

template <int LPC, int PPL, int CHUNK>
static void fill(KernelSet *k)
{
    k->cells_oci = (const void *)&k_cells<double, LPC, PPL, CHUNK, M_OCI>;
    k->cells_si = (const void *)&k_cells<double, LPC, PPL, CHUNK, M_SI>;
    k->commit_oci = (const void *)&k_percell<double, LPC, PPL, C_COMMIT_OCI>;
    k->commit_si = (const void *)&k_percell<double, LPC, PPL, C_COMMIT_SI>;
    k->si_prep = (const void *)&k_percell<double, LPC, PPL, C_SI_PREP>;
    k->guess = (const void *)&k_percell<double, LPC, PPL, C_GUESS>;
    k->march = (const void *)&k_si_march<double>;
    k->scan_reduce = (const void *)&k_scan_reduce<double>;
    k->scan_segments = (const void *)&k_scan_segments<double>;
    k->scan_apply = (const void *)&k_scan_apply<double>;
    k->be_cells = (const void *)&k_be_cells<double>;
    k->be_commit = (const void *)&k_be_commit<double>;
    k->lift_guess = (const void *)&k_lift<double, LPC, PPL, LIFT_GUESS>;
    k->lift_corr = (const void *)&k_lift<double, LPC, PPL, LIFT_CORR>;
    k->cells_oci_tma = nullptr;
    k->cells_oci_loop = nullptr;
    k->cells_si_tma = nullptr;
    k->cells_lin_tma = nullptr;
    k->commit_lin = nullptr;
    k->refine = nullptr;
    k->tma_stages = 0;
    k->cells_per_warp = CHUNK * (32 / LPC);
    k->cells_per_warp_pc = 32 / LPC;
}

bool kernel_set_f64(int lpc, int ppl, KernelSet *out)
{
    switch (lpc * 16 + ppl) {
    case 1 * 16 + 1: fill<1, 1, 8>(out); return true;
    case 2 * 16 + 1: fill<2, 1, 8>(out); return true;
    case 4 * 16 + 1: fill<4, 1, 8>(out); return true;
    case 8 * 16 + 1: fill<8, 1, 8>(out); return true;
    case 16 * 16 + 1: fill<16, 1, 8>(out); return true;
    case 32 * 16 + 1: fill<32, 1, 8>(out); return true;
    case 32 * 16 + 2: fill<32, 2, 8>(out); return true;
    case 32 * 16 + 4: fill<32, 4, 4>(out); return true;
    default: return false;
    }
}

}  // namespace ocik
