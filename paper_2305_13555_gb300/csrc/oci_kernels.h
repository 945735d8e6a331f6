// Kernel table for one precision: host-side addresses of the template
// instantiations for a given (lanes per cell, pairs per lane) layout.
#pragma once
#include "oci_device.cuh"
#include "oci_be.cuh"

namespace ocik {

struct KernelSet {
    const void *cells_oci;   // k_cells<M_OCI>
    const void *cells_si;    // k_cells<M_SI>
    const void *commit_oci;  // k_percell<C_COMMIT_OCI>
    const void *commit_si;   // k_percell<C_COMMIT_SI>
    const void *si_prep;     // k_percell<C_SI_PREP>
    const void *guess;       // k_percell<C_GUESS>
    const void *march;       // k_si_march
    const void *scan_reduce, *scan_segments, *scan_apply;  // parallel-prefix SI sweep
    const void *be_cells, *be_commit;                      // backward-Euler iteration and commit
    const void *lift_guess;  // k_lift<LIFT_GUESS>
    const void *lift_corr;   // k_lift<LIFT_CORR>
    const void *cells_oci_tma;  // k_cells_tma<M_OCI> (FP32, even P) or nullptr
    const void *cells_oci_loop; // k_cells_tma<M_OCI, persistent loop> or nullptr
    const void *cells_si_tma;   // k_cells_tma<M_SI>
    int tma_stages;             // ring depth of the staged kernels
    int tma_chunk;              // cell rows per chunk of the staged kernels
    int tma_max_warps;          // their launch bound, in warps
    const void *cells_lin_tma;  // k_cells_tma<M_LIN> (FP32 refinement) or nullptr
    const void *commit_lin;     // k_percell<C_COMMIT_LIN>
    const void *refine;         // k_refine_residual
    int cells_per_warp;      // cells handled by one warp pass of k_cells (CHUNK * 32 / LPC)
    int cells_per_warp_pc;   // cells per warp of k_percell (32 / LPC)
};

// The staged FP32 OCI iteration with BF16 face storage (k_cells_tma HALO 1-3).
struct HaloKernels {
    const void *entry;  // one iteration, float faces in, BF16 out
    const void *loop;   // persistent loop, BF16 in and out, until ST_SWITCH
    const void *exit;   // one iteration, BF16 in, float out
};

// Returns false if (lpc, ppl) has no instantiation.
bool kernel_set_f32(int lpc, int ppl, KernelSet *out);
bool kernel_set_bf16(int lpc, int ppl, HaloKernels *out);
// The barrier-free persistent OCI loop (8-row chunks, 2-stage ring) or nullptr.
const void *kernel_async_loop(int lpc, int ppl);
// Shared-memory bytes per stage of the staged FP32 kernels for P pairs and
// chunks of `chunk` cell rows.
unsigned tma_stage_bytes(int lpc, int chunk, int P);
bool kernel_set_f64(int lpc, int ppl, KernelSet *out);

}  // namespace ocik
