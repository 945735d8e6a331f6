// Dense per-material inverse variant of the OCI iteration.
//
// The paper's CPU OCI solves, in every cell, the 4N x 4N system (A - S) psi = c
// of Sec. "One-Cell Inversion (OCI)" with a dense LU (LAPACK _gesv).  Here the
// inverse (A - S)^{-1} is formed once per material on the host (FP64
// Gauss-Jordan with partial pivoting) and every iteration is
//   C   = right-hand sides c of all cells          (k_dense_rhs)
//   Psi = (A - S)^{-1} C, one GEMM per material    (cuBLAS)
//   outgoing corners -> faces, phi = sum w psi,
//   residual and convergence                       (k_dense_out)
// with the same face / moment / state buffers as the Woodbury kernels, so the
// step's initial iterate, the commit kernel and the learned guess are shared.
//
// Row order of one cell's system: r = 8 p + 4 sigma + i, pair p (mu_p > 0 of
// the Gauss-Legendre set), sigma = 0 for +mu_p and 1 for -mu_p, and
// i = (k L, k R, k+1/2 L, k+1/2 R).  Per ordinate with signed mu,
// a = (|mu| + dx sigma_t) / 2, e = dx / (2 v dt), h = mu / 2, the balance
// block (the A^+ / A^- matrices of the SI section in this order) is
//   [  a    h    e    0 ]
//   [ -h    a    0    e ]
//   [ -2e   0   a+2e  h ]
//   [  0   -2e  -h   a+2e]
// and S couples the same component of all ordinates with s w_n,
// s = dx sigma_s / 4 (the S_{l,n} of the OCI section).
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "oci_dense.h"

namespace ocik {

template <typename R>
__global__ void __launch_bounds__(256) k_dense_rhs(const KParams<R> p, const int *__restrict__ perm, int ncols,
                                                   R *__restrict__ C)
{
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const int iter = p.st->iter, base = p.st->base;
    const int frd = (base + iter) & 1;
    const r2<R> *fPr = p.faceP[frd], *fMr = p.faceM[frd];
    const int J = p.J, P = p.P;
    for (int col = w0; col < ncols; col += nw) {
        const int cell = perm[col];
        const r4<R> qd = p.cellq[cell];
        const R e = p.matpar[p.mat[cell]].x;
        R *c = C + (size_t)col * 8 * P;
        for (int pp = lane; pp < P; pp += 32) {
            const R mu = p.muw[pp].x;
            // incident corners: +mu from the left face, -mu from the right face
            const r2<R> inP = (p.bc_left == BC_REFLECT && cell == 0) ? fMr[pp] : fPr[(size_t)cell * P + pp];
            const r2<R> inM = (p.bc_right == BC_REFLECT && cell == J - 1) ? fPr[(size_t)J * P + pp]
                                                                           : fMr[(size_t)(cell + 1) * P + pp];
            const r4<R> pe = p.psi_edge[(size_t)cell * P + pp];  // (+L, +R, -L, -R) at t_{k-1/2}
            r4<R> *cp = reinterpret_cast<r4<R> *>(c + 8 * pp);
            cp[0] = r4<R>{qd.x + e * pe.x + mu * inP.x, qd.y + e * pe.y, qd.z + mu * inP.y, qd.w};
            cp[1] = r4<R>{qd.x + e * pe.z, qd.y + e * pe.w + mu * inM.x, qd.z, qd.w + mu * inM.y};
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_dense_out(const KParams<R> p, const int *__restrict__ perm, int ncols,
                                                   const R *__restrict__ Psi)
{
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const int iter = p.st->iter, base = p.st->base;
    const int fwr = ((base + iter) & 1) ^ 1;
    r2<R> *fPw = p.faceP[fwr], *fMw = p.faceM[fwr];
    const phi_t<R> *phr = iter == 0 ? p.phi0 : p.phi[iter & 1];
    phi_t<R> *phw = p.phi[(iter + 1) & 1];
    const int P = p.P;
    double d2 = 0.0, p2 = 0.0;
    for (int col = w0; col < ncols; col += nw) {
        const int cell = perm[col];
        const R *ps = Psi + (size_t)col * 8 * P;
        R m[4] = {0, 0, 0, 0};
        for (int pp = lane; pp < P; pp += 32) {
            const r4<R> a = reinterpret_cast<const r4<R> *>(ps + 8 * pp)[0];  // +mu_p
            const r4<R> b = reinterpret_cast<const r4<R> *>(ps + 8 * pp)[1];  // -mu_p
            const R w = p.muw[pp].y;
            m[0] += w * (a.x + b.x);
            m[1] += w * (a.y + b.y);
            m[2] += w * (a.z + b.z);
            m[3] += w * (a.w + b.w);
            fPw[(size_t)(cell + 1) * P + pp] = r2<R>{a.y, a.w};  // +mu leaves through the right face (corner R)
            fMw[(size_t)cell * P + pp] = r2<R>{b.x, b.z};        // -mu leaves through the left face (corner L)
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m[c] += __shfl_xor_sync(FULL, m[c], o);
        if (lane < 4) {
            const double phi = (double)m[lane];
            const double d = phi - PhiStore<R>::wide(phr[4 * (size_t)cell + lane]);
            d2 += d * d;
            p2 += phi * phi;
            phw[4 * (size_t)cell + lane] = phi_from_double<R>(phi);
        }
    }
    finalize_iteration(d2, p2, p.partials, p.st, p.cfg, iter, 0, p.cond);
}

namespace {

// Inverse of the n x n row-major matrix a (overwritten) into inv, by
// Gauss-Jordan elimination with partial pivoting.  False if singular.
bool invert(std::vector<double> &a, std::vector<double> &inv, int n)
{
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = std::fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(a[(size_t)i * n + k]) > best) { best = std::fabs(a[(size_t)i * n + k]); piv = i; }
        if (!(best > 0.0) || !std::isfinite(best)) return false;
        if (piv != k)
            for (int j = 0; j < n; ++j) {
                std::swap(a[(size_t)k * n + j], a[(size_t)piv * n + j]);
                std::swap(inv[(size_t)k * n + j], inv[(size_t)piv * n + j]);
            }
        const double d = 1.0 / a[(size_t)k * n + k];
        for (int j = 0; j < n; ++j) { a[(size_t)k * n + j] *= d; inv[(size_t)k * n + j] *= d; }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            const double f = a[(size_t)i * n + k];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                a[(size_t)i * n + j] -= f * a[(size_t)k * n + j];
                inv[(size_t)i * n + j] -= f * inv[(size_t)k * n + j];
            }
        }
    }
    return true;
}

}  // namespace

bool dense_inverse(const double *mu_p, const double *w_p, int P, double dx, double sigma_t, double sigma_s,
                   double e, std::vector<double> &inv)
{
    const int n = 8 * P;
    std::vector<double> a((size_t)n * n, 0.0);
    const double s = dx * sigma_s / 4.0;
    for (int p = 0; p < P; ++p)
        for (int sg = 0; sg < 2; ++sg) {
            const double mu = sg == 0 ? mu_p[p] : -mu_p[p];
            const double aa = (std::fabs(mu) + dx * sigma_t) / 2.0, h = mu / 2.0;
            const double blk[4][4] = {{aa, h, e, 0.0}, {-h, aa, 0.0, e}, {-2.0 * e, 0.0, aa + 2.0 * e, h},
                                      {0.0, -2.0 * e, -h, aa + 2.0 * e}};
            const int r0 = 8 * p + 4 * sg;
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) a[(size_t)(r0 + i) * n + r0 + j] = blk[i][j];
        }
    for (int ro = 0; ro < 2 * P; ++ro)       // ordinate of the row
        for (int co = 0; co < 2 * P; ++co)   // ordinate of the column
            for (int i = 0; i < 4; ++i) a[(size_t)(4 * ro + i) * n + 4 * co + i] -= s * w_p[co / 2];
    return invert(a, inv, n);
}

template <typename R>
int dense_iteration(const KParams<R> &p, const DenseBuffers &d, int grid, cudaStream_t s)
{
    void *a_rhs[] = {const_cast<KParams<R> *>(&p), const_cast<int **>(&d.perm), const_cast<int *>(&d.ncols),
                     const_cast<void **>(&d.C)};
    if (cudaLaunchKernel((const void *)&k_dense_rhs<R>, dim3(grid), dim3(256), a_rhs, 0, s) != cudaSuccess)
        return 3;
    cublasHandle_t hb = static_cast<cublasHandle_t>(d.blas);
    if (cublasSetStream(hb, s) != CUBLAS_STATUS_SUCCESS) return 3;
    const int n = 8 * p.P;
    for (size_t m = 0; m < d.col_off.size() - 1; ++m) {
        const int c0 = d.col_off[m], nc = d.col_off[m + 1] - c0;
        if (nc == 0) continue;
        const R one = 1, zero = 0;
        const R *A = static_cast<const R *>(d.minv) + (size_t)m * n * n;
        const R *B = static_cast<const R *>(d.C) + (size_t)c0 * n;
        R *Cc = static_cast<R *>(d.Psi) + (size_t)c0 * n;
        // row-major inverse = column-major transpose: Psi = op_T(A) * B
        cublasStatus_t st;
        if constexpr (sizeof(R) == 8)
            st = cublasDgemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, n, nc, n, &one, A, n, B, n, &zero, Cc, n);
        else
            st = cublasSgemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, n, nc, n, &one, A, n, B, n, &zero, Cc, n);
        if (st != CUBLAS_STATUS_SUCCESS) return 3;
    }
    void *a_out[] = {const_cast<KParams<R> *>(&p), const_cast<int **>(&d.perm), const_cast<int *>(&d.ncols),
                     const_cast<void **>(&d.Psi)};
    if (cudaLaunchKernel((const void *)&k_dense_out<R>, dim3(grid), dim3(256), a_out, 0, s) != cudaSuccess)
        return 3;
    return 0;
}

template int dense_iteration<double>(const KParams<double> &, const DenseBuffers &, int, cudaStream_t);
template int dense_iteration<float>(const KParams<float> &, const DenseBuffers &, int, cudaStream_t);

int dense_blas_create(void **out)
{
    cublasHandle_t hb;
    if (cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS) return 3;
    *out = hb;
    return 0;
}

void dense_blas_destroy(void *b)
{
    if (b) cublasDestroy(static_cast<cublasHandle_t>(b));
}

}  // namespace ocik
