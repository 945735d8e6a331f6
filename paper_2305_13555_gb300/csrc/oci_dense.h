// Dense per-material inverse variant of the OCI iteration (oci_dense.cu).
#pragma once
#include <vector>

#include "oci_device.cuh"

namespace ocik {

struct DenseBuffers {
    void *blas = nullptr;           // cublasHandle_t
    void *mem = nullptr;            // one device allocation for the arrays below
    void *minv = nullptr;           // [n_mat][8P][8P] row-major (A - S)^{-1}, storage precision
    void *C = nullptr, *Psi = nullptr;  // [J][8P] right-hand sides / solutions, cells grouped by material
    int *perm = nullptr;            // [J] cell of each column
    int ncols = 0;
    std::vector<int> col_off;       // [n_mat + 1] first column of each material
};

// (A - S)^{-1} of one material in the row order of oci_dense.cu, FP64.
bool dense_inverse(const double *mu_p, const double *w_p, int P, double dx, double sigma_t, double sigma_s,
                   double e, std::vector<double> &inv);

// One iteration: right-hand sides, per-material GEMMs, outgoing corners,
// moments and the residual (finalised on the device).  0 or OCI_ECUDA (3).
template <typename R>
int dense_iteration(const KParams<R> &p, const DenseBuffers &d, int grid, cudaStream_t s);

int dense_blas_create(void **out);
void dense_blas_destroy(void *b);

}  // namespace ocik
