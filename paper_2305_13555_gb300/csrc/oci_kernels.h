// Kernel table for one precision: host-side addresses of the template
// instantiations for a given (lanes per cell, pairs per lane) layout.
#pragma once
#include "oci_device.cuh"

namespace ocik {

struct KernelSet {
    const void *cells_oci;   // k_cells<M_OCI>
    const void *cells_si;    // k_cells<M_SI>
    const void *commit_oci;  // k_percell<C_COMMIT_OCI>
    const void *commit_si;   // k_percell<C_COMMIT_SI>
    const void *si_prep;     // k_percell<C_SI_PREP>
    const void *guess;       // k_percell<C_GUESS>
    const void *march;       // k_si_march
    int cells_per_warp;      // cells handled by one warp pass of k_cells (CHUNK * 32 / LPC)
    int cells_per_warp_pc;   // cells per warp of k_percell (32 / LPC)
};

// Returns false if (lpc, ppl) has no instantiation.
bool kernel_set_f32(int lpc, int ppl, KernelSet *out);
bool kernel_set_f64(int lpc, int ppl, KernelSet *out);

}  // namespace ocik
