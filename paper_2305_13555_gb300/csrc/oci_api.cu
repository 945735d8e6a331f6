// C ABI of the one-cell-inversion library (declarations and contracts in
// include/oci.h).  Host-side setup in double precision: Gauss-Legendre set,
// per-material block inverses and Woodbury capacitance; device memory owned by
// the handle; each time step is one CUDA graph launch, so the host
// synchronises once per step.  Inside the graph the iterations run either in
// one persistent cooperative launch (the staged FP32 kernel: it loops until the
// step is decided) or as a device-side conditional WHILE node around one
// launch per iteration (FP64, SI, backward Euler, the FP32 refinement).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/oci.h"
#include "oci_dense.h"
#include "oci_kernels.h"

using ocik::IterConfig;
using ocik::IterState;
using ocik::KernelSet;
using ocik::KParams;
using ocik::kmat;
using ocik::r2;
using ocik::r4;

namespace {

constexpr int kBlock = 256;

// Gauss-Legendre nodes (ascending) and weights by Newton's method on P_N,
// P_N' from N (x P_N - P_{N-1}) / (x^2 - 1), started from the Tricomi
// asymptotic estimate of the k-th root.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.141592653589793238462643;
    for (int k = 1; k <= n / 2 + (n & 1); ++k) {
        const double th = pi * (4.0 * k - 1.0) / (4.0 * n + 2.0);
        double r = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(th);
        double d = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1.0, pc = r;  // P_0, P_1
            for (int l = 2; l <= n; ++l) {
                const double pn = ((2.0 * l - 1.0) * r * pc - (l - 1.0) * pm) / l;
                pm = pc;
                pc = pn;
            }
            if (n == 1) { pm = 1.0; pc = r; }
            d = n * (r * pc - pm) / (r * r - 1.0);
            const double step = pc / d;
            r -= step;
            if (std::fabs(step) <= 4e-17) break;
        }
        double pm = 1.0, pc = r;
        for (int l = 2; l <= n; ++l) {
            const double pn = ((2.0 * l - 1.0) * r * pc - (l - 1.0) * pm) / l;
            pm = pc;
            pc = pn;
        }
        if (n == 1) { pm = 1.0; pc = r; }
        d = n * (r * pc - pm) / (r * r - 1.0);
        const double wk = 2.0 / ((1.0 - r * r) * d * d);
        x[n - k] = r;   // k-th largest
        x[k - 1] = -r;
        w[n - k] = wk;
        w[k - 1] = wk;
    }
    if (n & 1) x[n / 2] = 0.0;
}

struct Material {
    double dx, st, ss;
};

}  // namespace

struct oci_handle {
    int J = 0, N = 0, P = 0, prec = 0, bcl = 0, bcr = 0;
    double v = 1.0, dt = 1.0;
    int lpc = 32, ppl = 1;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<double> mu, w;      // full N ordinates
    std::vector<double> dx;         // per cell
    std::vector<int> mat;           // per cell
    std::vector<Material> mats;
    KernelSet ks{};
    // device memory (one allocation)
    void *d_base = nullptr;
    size_t d_bytes = 0;
    void *faceP[3] = {nullptr, nullptr, nullptr}, *faceM[3] = {nullptr, nullptr, nullptr};  // [2]: barrier-free loop
    void *psi_edge = nullptr, *g = nullptr, *cellq = nullptr, *tab = nullptr, *matpar = nullptr, *muw = nullptr,
         *refl = nullptr;
    int *d_mat = nullptr;
    kmat *d_matK = nullptr;
    void *d_matKf = nullptr;        // FP32 mode: capacitance as double-float pairs
    double *phi[2] = {nullptr, nullptr}, *phi0 = nullptr, *phi_out = nullptr, *partials = nullptr;
    IterState *d_st = nullptr;
    IterConfig *d_cfg = nullptr;
    IterState *h_st = nullptr;      // pinned
    IterConfig cfg{};
    IterConfig cfg_dev{};            // what the device copy holds
    int grid_cells = 1, grid_pc = 1;
    // iteration kernels actually launched (staged TMA variant when available)
    const void *cells_oci = nullptr, *cells_si = nullptr, *cells_lin = nullptr;
    int cells_grid = 1, cells_block = 256;
    unsigned cells_smem = 0;
    bool staged = false;
    // graphs
    cudaGraph_t graph_oci = nullptr, graph_si = nullptr;
    cudaGraphExec_t exec_oci = nullptr, exec_si = nullptr;
    bool guess_valid = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err;
    // learned guess
    int nn_mode = OCI_NN_OFF, nn_kcorr = 50;
    // OCI_NN_GUESS_ADAPTIVE: position in the plain/guessed/guessed/plain trial,
    // iterations of its plain and guessed steps, and the current choice
    int nn_trial = 0;
    long nn_trial_plain = 0, nn_trial_nn = 0;
    bool nn_use = true;
    int nn_since_trial = 0;
    void *nn_mem = nullptr;          // one allocation for everything below
    float *nn_params = nullptr, *nn_in = nullptr, *nn_out = nullptr, *nn_scale = nullptr, *nn_stat = nullptr,
          *nn_qfeat = nullptr;
    double *nn_phat = nullptr, *nn_hist[2] = {nullptr, nullptr}, *nn_phi_bak = nullptr;
    void *nn_ws = nullptr, *nn_face_bak = nullptr;
    size_t nn_ws_bytes = 0;
    cudaGraph_t graph_cont = nullptr;
    cudaGraphExec_t exec_cont = nullptr;
    std::vector<double> q_host;      // sources (for the network's inputs; valid while q_host_valid)
    bool q_host_valid = false;
    double *q_dev = nullptr, *dx_dev = nullptr;  // FP64 source moments [J][4] and cell widths [J]
    // backward-Euler time scheme (oci_set_time_scheme)
    int scheme = OCI_TIME_MB;
    void *be_mem = nullptr;          // 1/t per material and pair (storage precision), K per material (FP64)
    void *be_tab = nullptr;
    double *be_K = nullptr;
    float2 *be_Kf = nullptr;
    cudaGraph_t graph_be = nullptr;
    cudaGraphExec_t exec_be = nullptr;
    std::vector<double> bc_left_host, bc_right_host;  // prescribed incident data
    // FP32 refinement (stalled steps): FP64 tables, saved halo, residual, phi(h0)
    double *ref_tab = nullptr, *ref_par = nullptr, *ref_muw = nullptr;
    void *ref_h0P = nullptr, *ref_h0M = nullptr, *ref_r0 = nullptr, *ref_phi = nullptr;
    cudaGraph_t graph_lin = nullptr;
    cudaGraphExec_t exec_lin = nullptr;
    int refinements = 0;
    // dense per-material inverse variant (oci_set_solver)
    int solver = OCI_SOLVER_WOODBURY;
    ocik::DenseBuffers dense;
    int dense_grid = 1;
    // SI sweep as a parallel prefix (oci_set_sweep)
    int sweep = OCI_SWEEP_MARCH;
    bool pdl_graph = true;           // programmatic edges between iterations (cleared if unsupported)
    // persistent OCI loop (staged FP32 kernel, cooperative launch): one launch per step
    const void *cells_loop = nullptr;
    bool use_loop = false;
    double *loop_partials = nullptr;
    unsigned *loop_bar = nullptr;
    int loop_fixed = 0;
    void *scan_mem = nullptr;  // segment maps [2P][nseg], entering values [2P][nseg]
    int scan_nseg = 0;
    // BF16 halo (oci_set_halo): face buffers as bf16 pairs and the step graph
    // entry -> BF16 loop -> exit -> FP32 loop -> commit
    int halo = OCI_HALO_FP32;
    ocik::HaloKernels hk{};
    void *hface_mem = nullptr;
    unsigned *hfP[2] = {nullptr, nullptr}, *hfM[2] = {nullptr, nullptr};
    cudaGraph_t graph_oci_h = nullptr;
    cudaGraphExec_t exec_oci_h = nullptr;
    // barrier-free persistent OCI loop (staged FP32, S_32 / S_64 / S_128): its
    // kernel, third face buffer pair, sync block + per-warp counts (zeroed per
    // launch) and per-warp partials; the barrier loop's graph kept for the corrector
    bool use_async = false;
    const void *cells_async = nullptr;
    void *async_mem = nullptr;
    ocik::AsyncSync *as = nullptr;
    unsigned *as_done = nullptr;
    double *as_part = nullptr;
    size_t as_zero_bytes = 0;
    cudaGraph_t graph_oci_bar = nullptr;
    cudaGraphExec_t exec_oci_bar = nullptr;
    // pipelined stepping (oci_step_async / oci_step_wait): a copy stream for the
    // next step's source and the last step's moments, two device snapshots of
    // the moments, and the events ordering them against the handle's stream
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_done = nullptr, ev_q_ready = nullptr, ev_q_free = nullptr, ev_snap[2] = {nullptr, nullptr},
                ev_d2h[2] = {nullptr, nullptr};
    double *phi_snap[2] = {nullptr, nullptr};
    // domain decomposition (oci_dd_*): a step driven one iteration at a time
    bool dd_active = false;
    int dd_iter = 0;
    int snap_k = 0;
    bool step_pending = false, q_pending = false;
    bool pend_halo = false, pend_async = false;
    int pend_launches = 0;
    // several steps in one call (oci_run_steps): the sources staged on an upload
    // stream into two device buffers (each kept until the step two after its own
    // is enqueued, so a step's cell sources can be scaled again); per-slot state
    // copies (pinned) and events
    void *rs_mem = nullptr;
    double *rs_stage[2] = {nullptr, nullptr};
    IterState *rs_st = nullptr;
    cudaStream_t rs_up = nullptr;  // uploads, apart from the copy stream's downloads (which wait for their steps)
    cudaEvent_t rs_ev0[2] = {nullptr, nullptr}, rs_ev1[2] = {nullptr, nullptr}, rs_done[2] = {nullptr, nullptr},
                rs_ready[2] = {nullptr, nullptr}, rs_free[2] = {nullptr, nullptr};
};

namespace {

int cuda_fail(oci_handle *h, cudaError_t e, const char *what)
{
    if (h) {
        char buf[256];
        std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
        h->err = buf;
    }
    return OCI_ECUDA;
}

#define CK(h, call)                                          \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

size_t rsize(const oci_handle *h) { return h->prec == OCI_FP64 ? 8 : 4; }

template <typename R>
KParams<R> make_params(const oci_handle *h, int use_cond, cudaGraphConditionalHandle cond)
{
    KParams<R> p{};
    p.J = h->J;
    p.P = h->P;
    p.bc_left = h->bcl;
    p.bc_right = h->bcr;
    p.use_cond = use_cond;
    p.cond = cond;
    p.mat = h->d_mat;
    p.cellq = (const r4<R> *)h->cellq;
    p.tab = (const r4<R> *)h->tab;
    p.matpar = (const r2<R> *)h->matpar;
    p.matK = h->d_matK;
    p.muw = (const r2<R> *)h->muw;
    for (int b = 0; b < 2; ++b) {
        p.faceP[b] = (r2<R> *)h->faceP[b];
        p.faceM[b] = (r2<R> *)h->faceM[b];
        p.phi[b] = (ocik::phi_t<R> *)h->phi[b];
    }
    p.faceP[2] = (r2<R> *)h->faceP[2];
    p.faceM[2] = (r2<R> *)h->faceM[2];
    p.as = h->as;
    p.as_done = h->as_done;
    p.as_part = h->as_part;
    p.psi_edge = (r4<R> *)h->psi_edge;
    p.g = (r4<R> *)h->g;
    p.refl = (r2<R> *)h->refl;
    p.phi0 = (ocik::phi_t<R> *)h->phi0;
    p.phi_out = h->phi_out;
    p.matKf = (const float4 *)h->d_matKf;
    p.h0P = (const r2<R> *)h->ref_h0P;
    p.h0M = (const r2<R> *)h->ref_h0M;
    p.r0 = (const r4<R> *)h->ref_r0;
    p.phi_ref = (const float2 *)h->ref_phi;
    p.partials = h->partials;
    p.st = h->d_st;
    p.cfg = h->d_cfg;
    p.loop_partials = h->loop_partials;
    p.loop_bar = h->loop_bar;
    p.loop_fixed = h->loop_fixed;
    for (int b = 0; b < 2; ++b) {
        p.hfP[b] = h->hfP[b];
        p.hfM[b] = h->hfM[b];
    }
    return p;
}

// Upload a host array converted to the storage precision.
int upload_real(oci_handle *h, void *dst, const std::vector<double> &src)
{
    if (h->prec == OCI_FP64) {
        CK(h, cudaMemcpyAsync(dst, src.data(), src.size() * 8, cudaMemcpyHostToDevice, h->stream));
    } else {
        std::vector<float> f(src.begin(), src.end());
        CK(h, cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));  // f is a temporary
        return OCI_OK;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return OCI_OK;
}

// psi [J][N][2] (device copy, ordinates ascending) -> psi_edge [J][P]
// (+L, +R, -L, -R) and phi = (sum w psi_L, sum w psi_R) in both time moments:
// one warp per cell, lanes over ordinate pairs, the moments summed in FP64
// (w_p is the weight of both +mu_p and -mu_p; Gauss-Legendre is symmetric).
template <typename R>
__global__ void k_load_state(const double *__restrict__ psi, const double *__restrict__ wpos, int J, int P,
                             r4<R> *psi_edge, ocik::phi_t<R> *phi0, double *phi_out)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = gw; j < J; j += nw) {
        const double *pj = psi + (size_t)j * P * 4;
        double sL = 0.0, sR = 0.0;
        for (int p = lane; p < P; p += 32) {
            const double2 a = *(const double2 *)(pj + 2 * (P + p));      // +mu_p
            const double2 b = *(const double2 *)(pj + 2 * (P - 1 - p));  // -mu_p
            psi_edge[(size_t)j * P + p] = r4<R>{(R)a.x, (R)a.y, (R)b.x, (R)b.y};
            sL += wpos[p] * (a.x + b.x);
            sR += wpos[p] * (a.y + b.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sL += __shfl_xor_sync(0xffffffffu, sL, o);
            sR += __shfl_xor_sync(0xffffffffu, sR, o);
        }
        if (lane < 4) {
            const double f = (lane & 1) ? sR : sL;
            phi_out[4 * (size_t)j + lane] = f;
            phi0[4 * (size_t)j + lane] = ocik::phi_from_double<R>(f);
        }
    }
}

// New committed state from host psi [J][N][2] (nullptr: zero): one
// host-to-device copy into stream-ordered scratch (direct DMA when the caller's
// buffer is page-locked) and the conversion kernel.  The learned guess's flux
// history restarts from the new moments.
int load_state(oci_handle *h, const double *psi)
{
    const int J = h->J, P = h->P;
    const size_t rs = h->prec == OCI_FP64 ? 8 : 4;
    if (!psi) {
        CK(h, cudaMemsetAsync(h->psi_edge, 0, (size_t)J * P * 4 * rs, h->stream));
        CK(h, cudaMemsetAsync(h->phi0, 0, (size_t)J * 32, h->stream));  // double or float2 per moment
        CK(h, cudaMemsetAsync(h->phi_out, 0, (size_t)J * 32, h->stream));
    } else {
        const size_t n = (size_t)J * P * 4;
        std::vector<double> wpos(P);
        for (int p = 0; p < P; ++p) wpos[p] = h->w[P + p];
        double *scratch = nullptr;
        CK(h, cudaMallocAsync((void **)&scratch, (n + P) * 8, h->stream));
        cudaError_t e = cudaMemcpyAsync(scratch, psi, n * 8, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + n, wpos.data(), P * 8, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) {
            const int grid = std::max(1, std::min((J + 7) / 8, 152 * 8));
            if (h->prec == OCI_FP64)
                k_load_state<double><<<grid, 256, 0, h->stream>>>(scratch, scratch + n, J, P, (r4<double> *)h->psi_edge,
                                                                  (ocik::phi_t<double> *)h->phi0, h->phi_out);
            else
                k_load_state<float><<<grid, 256, 0, h->stream>>>(scratch, scratch + n, J, P, (r4<float> *)h->psi_edge,
                                                                 (ocik::phi_t<float> *)h->phi0, h->phi_out);
            e = cudaGetLastError();
        }
        const cudaError_t ef = cudaFreeAsync(scratch, h->stream);
        CK(h, e);
        CK(h, ef);
    }
    if (h->nn_hist[0]) {
        CK(h, cudaMemcpyAsync(h->nn_hist[0], h->phi_out, (size_t)J * 32, cudaMemcpyDeviceToDevice, h->stream));
        CK(h, cudaMemcpyAsync(h->nn_hist[1], h->phi_out, (size_t)J * 32, cudaMemcpyDeviceToDevice, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));  // wpos is a temporary; the call returns with the state in place
    h->guess_valid = false;
    return OCI_OK;
}

// Static network inputs per cell (see oci_nn.h) and the source input qfeat.
void nn_host_features(const oci_handle *h, std::vector<float> &stat, std::vector<float> &qf)
{
    const int J = h->J;
    const double vdt = std::isinf(h->v) ? 1.0 : h->v * h->dt;
    stat.assign((size_t)J * 4, 0.f);
    qf.assign(J, 0.f);
    for (int j = 0; j < J; ++j) {
        const Material &m = h->mats[h->mat[j]];
        const double st = std::max(m.st, 1e-30);
        stat[4 * j + 0] = (float)(0.5 * std::log10(st));
        stat[4 * j + 1] = (float)(m.st > 0.0 ? m.ss / m.st : 0.0);
        stat[4 * j + 2] = (float)std::log10(std::max(m.st * m.dx, 1e-30));
        stat[4 * j + 3] = (float)std::log10(std::max(m.st * vdt, 1e-30));
        if (!h->q_host.empty()) qf[j] = (float)(vdt * 0.5 * (h->q_host[4 * (size_t)j] + h->q_host[4 * (size_t)j + 1]));
    }
}

// (dx/4) Q in the storage precision, from the FP64 source moments on the device.
template <typename R>
__global__ void k_scale_source(const double *__restrict__ q, const double *__restrict__ dx, int J, r4<R> *cellq)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < J; j += gridDim.x * blockDim.x) {
        const double f = dx[j] / 4.0;
        const double *qj = q + 4 * (size_t)j;
        cellq[j] = r4<R>{(R)(f * qj[0]), (R)(f * qj[1]), (R)(f * qj[2]), (R)(f * qj[3])};
    }
}

// The host keeps a copy of Q only while a network is attached (its source input).
int sync_q_host(oci_handle *h)
{
    if (h->q_host_valid) return OCI_OK;
    h->q_host.resize((size_t)h->J * 4);
    CK(h, cudaMemcpyAsync(h->q_host.data(), h->q_dev, (size_t)h->J * 32, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->q_host_valid = true;
    return OCI_OK;
}

// New source moments: one host-to-device copy of Q and a scaling kernel, no
// host-side conversion (the copy is enqueued; pageable sources are staged by
// the driver before the call returns).
int upload_source(oci_handle *h, const double *q)
{
    const size_t bytes = (size_t)h->J * 32;
    if (q) CK(h, cudaMemcpyAsync(h->q_dev, q, bytes, cudaMemcpyHostToDevice, h->stream));
    else CK(h, cudaMemsetAsync(h->q_dev, 0, bytes, h->stream));
    const int grid = std::min((h->J + 255) / 256, 152 * 8);
    if (h->prec == OCI_FP64)
        k_scale_source<double><<<grid, 256, 0, h->stream>>>(h->q_dev, h->dx_dev, h->J, (r4<double> *)h->cellq);
    else
        k_scale_source<float><<<grid, 256, 0, h->stream>>>(h->q_dev, h->dx_dev, h->J, (r4<float> *)h->cellq);
    CK(h, cudaGetLastError());
    if (h->ev_q_free) CK(h, cudaEventRecord(h->ev_q_free, h->stream));  // q_dev consumed
    h->q_host_valid = false;
    if (h->nn_mem) {
        if (q) {
            h->q_host.assign(q, q + (size_t)h->J * 4);
            h->q_host_valid = true;
        } else {
            h->q_host.assign((size_t)h->J * 4, 0.0);
            h->q_host_valid = true;
        }
        std::vector<float> st, qf;
        nn_host_features(h, st, qf);
        CK(h, cudaMemcpyAsync(h->nn_qfeat, qf.data(), sizeof(float) * qf.size(), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return OCI_OK;
}

// Pipelined stepping: the copy stream, events and moment snapshots (once).
int pipe_setup(oci_handle *h)
{
    if (h->copy_stream) return OCI_OK;
    CK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&h->ev_done, &h->ev_q_ready, &h->ev_q_free, &h->ev_snap[0], &h->ev_snap[1], &h->ev_d2h[0],
                           &h->ev_d2h[1]})
        CK(h, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    for (int k = 0; k < 2; ++k)
        if (cudaMalloc((void **)&h->phi_snap[k], (size_t)h->J * 32) != cudaSuccess) return OCI_ENOMEM;
    return OCI_OK;
}

// A source staged on the copy stream while a step was running: scale it into
// the cell sources ahead of the next step.
int apply_pending_source(oci_handle *h)
{
    if (!h->q_pending) return OCI_OK;
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_q_ready, 0));
    const int grid = std::min((h->J + 255) / 256, 152 * 8);
    if (h->prec == OCI_FP64)
        k_scale_source<double><<<grid, 256, 0, h->stream>>>(h->q_dev, h->dx_dev, h->J, (r4<double> *)h->cellq);
    else
        k_scale_source<float><<<grid, 256, 0, h->stream>>>(h->q_dev, h->dx_dev, h->J, (r4<float> *)h->cellq);
    CK(h, cudaGetLastError());
    CK(h, cudaEventRecord(h->ev_q_free, h->stream));
    h->q_pending = false;
    h->q_host_valid = false;
    return OCI_OK;
}

// Per-material tables: complex entries of A_{+mu_p}^{-1}, (e, s), and the
// capacitance inverse K = (I - s M_r)^{-1}, M_r = sum_p 2 w_p Re(A_p^{-1}).
int build_tables(oci_handle *h)
{
    const int P = h->P, nm = (int)h->mats.size();
    std::vector<double> tab((size_t)nm * P * 8), par((size_t)nm * 2), muw((size_t)P * 2);
    std::vector<kmat> K(nm);
    const bool steady = std::isinf(h->v);
    for (int p = 0; p < P; ++p) {
        muw[2 * p] = h->mu[P + p];
        muw[2 * p + 1] = h->w[P + p];
    }
    for (int m = 0; m < nm; ++m) {
        const Material &mt = h->mats[m];
        const double e = steady ? 0.0 : mt.dx / (2.0 * h->v * h->dt);
        const double s = mt.dx * mt.ss / 4.0;
        double M00 = 0, M01 = 0, M10 = 0, M11 = 0;
        for (int p = 0; p < P; ++p) {
            const double mu = h->mu[P + p];
            const std::complex<double> t((mu + mt.dx * mt.st) / 2.0, -mu / 2.0);
            const std::complex<double> D = t * (t + 2.0 * e) + 2.0 * e * e;
            const std::complex<double> Pc = (t + 2.0 * e) / D, Rc = -e / D, Uc = 2.0 * e / D, Vc = t / D;
            double *o = &tab[((size_t)m * P + p) * 8];
            o[0] = Pc.real(); o[1] = Pc.imag(); o[2] = Rc.real(); o[3] = Rc.imag();
            o[4] = Uc.real(); o[5] = Uc.imag(); o[6] = Vc.real(); o[7] = Vc.imag();
            const double wp = 2.0 * h->w[P + p];
            M00 += wp * Pc.real(); M01 += wp * Rc.real(); M10 += wp * Uc.real(); M11 += wp * Vc.real();
        }
        const double a00 = 1.0 - s * M00, a01 = -s * M01, a10 = -s * M10, a11 = 1.0 - s * M11;
        const double det = a00 * a11 - a01 * a10;
        if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return OCI_EINVAL;
        K[m] = kmat{a11 / det, -a01 / det, -a10 / det, a00 / det};
        par[2 * m] = e;
        par[2 * m + 1] = s;
    }
    int rc = upload_real(h, h->tab, tab);
    if (!rc) rc = upload_real(h, h->matpar, par);
    if (!rc) rc = upload_real(h, h->muw, muw);
    if (rc) return rc;
    if (h->ref_tab) {  // FP64 copies for the refinement's residual pass
        CK(h, cudaMemcpy(h->ref_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
        CK(h, cudaMemcpy(h->ref_par, par.data(), sizeof(double) * par.size(), cudaMemcpyHostToDevice));
        CK(h, cudaMemcpy(h->ref_muw, muw.data(), sizeof(double) * muw.size(), cudaMemcpyHostToDevice));
    }
    CK(h, cudaMemcpy(h->d_matK, K.data(), sizeof(kmat) * nm, cudaMemcpyHostToDevice));
    {
        std::vector<float> kf((size_t)nm * 8);
        for (int m = 0; m < nm; ++m) {
            const double k[4] = {K[m].k00, K[m].k01, K[m].k10, K[m].k11};
            for (int i = 0; i < 4; ++i) {
                kf[(size_t)m * 8 + 2 * i] = (float)k[i];
                kf[(size_t)m * 8 + 2 * i + 1] = (float)(k[i] - (double)(float)k[i]);
            }
        }
        CK(h, cudaMemcpy(h->d_matKf, kf.data(), sizeof(float) * kf.size(), cudaMemcpyHostToDevice));
    }
    CK(h, cudaMemcpy(h->d_mat, h->mat.data(), sizeof(int) * h->J, cudaMemcpyHostToDevice));
    return OCI_OK;
}

int upload_boundaries(oci_handle *h, const double *bl, const double *br)
{
    if (bl && bl != h->bc_left_host.data()) h->bc_left_host.assign(bl, bl + (size_t)h->P * 2);
    if (br && br != h->bc_right_host.data()) h->bc_right_host.assign(br, br + (size_t)h->P * 2);
    const int J = h->J, P = h->P;
    const size_t rs = rsize(h);
    std::vector<double> l((size_t)P * 2, 0.0), r((size_t)P * 2, 0.0);
    if (h->bcl == OCI_BC_INCIDENT && bl) std::memcpy(l.data(), bl, sizeof(double) * P * 2);
    if (h->bcr == OCI_BC_INCIDENT && br) std::memcpy(r.data(), br, sizeof(double) * P * 2);
    for (int b = 0; b < (h->faceP[2] ? 3 : 2); ++b) {
        int rc = upload_real(h, h->faceP[b], l);  // face 0 = first P pairs
        if (rc) return rc;
        rc = upload_real(h, (char *)h->faceM[b] + (size_t)J * P * 2 * rs, r);  // face J
        if (rc) return rc;
    }
    return OCI_OK;
}

// Kernel node helper.
int add_kernel(oci_handle *h, cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *dep, int ndep,
               const void *fn, dim3 grid, dim3 block, void **args, unsigned smem = 0)
{
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeKernel;
    np.kernel.func = const_cast<void *>(fn);
    np.kernel.gridDim = grid;
    np.kernel.blockDim = block;
    np.kernel.sharedMemBytes = smem;
    np.kernel.kernelParams = args;
    CK(h, cudaGraphAddNode(node, g, dep, nullptr, ndep, &np));
    return OCI_OK;
}

// The OCI iteration inside a WHILE body: with the staged kernel, kUnroll
// launches chained by programmatic edges (each iteration's prologue and
// iteration-invariant copies overlap the previous one's tail; launches after
// the step has ended return at once), else one launch.
constexpr int kUnroll = 4;

int add_iterations(oci_handle *h, cudaGraph_t body, const void *fn, void **args)
{
    const int n = (h->staged && h->pdl_graph) ? kUnroll : 1;
    cudaGraphNode_t prev = nullptr;
    for (int i = 0; i < n; ++i) {
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeKernel;
        np.kernel.func = const_cast<void *>(fn);
        np.kernel.gridDim = dim3(h->cells_grid);
        np.kernel.blockDim = dim3(h->cells_block);
        np.kernel.sharedMemBytes = h->cells_smem;
        np.kernel.kernelParams = args;
        cudaGraphEdgeData ed{};
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.type = cudaGraphDependencyTypeProgrammatic;
        cudaGraphNode_t node;
        CK(h, cudaGraphAddNode(&node, body, i ? &prev : nullptr, i ? &ed : nullptr, i ? 1 : 0, &np));
        prev = node;
    }
    return OCI_OK;
}

// The persistent OCI loop in a graph: zero the barrier counter, then one
// cooperative launch that iterates until the step is decided (or paused).
int add_loop(oci_handle *h, cudaGraph_t g, const cudaGraphNode_t *dep, cudaGraphNode_t *out, void **args)
{
    cudaMemsetParams mp{};
    mp.dst = h->loop_bar;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned);
    mp.width = 1;
    mp.height = 1;
    cudaGraphNode_t n_zero;
    CK(h, cudaGraphAddMemsetNode(&n_zero, g, dep, dep ? 1 : 0, &mp));
    int rc = add_kernel(h, g, out, &n_zero, 1, h->cells_loop, dim3(h->cells_grid), dim3(h->cells_block), args,
                        h->cells_smem);
    if (rc) return rc;
    cudaLaunchAttributeValue v{};
    v.cooperative = 1;
    CK(h, cudaGraphKernelNodeSetAttribute(*out, cudaLaunchAttributeCooperative, &v));
    return OCI_OK;
}

// Step graph: begin -> [si_prep] -> WHILE { [march ->] cells } -> commit
// (OCI with the persistent loop: begin -> loop, which ends the step itself).
template <typename R>
int build_graph(oci_handle *h, bool si, cudaGraph_t *gout, cudaGraphExec_t *eout, bool bar_loop = false)
{
    cudaGraph_t g;
    CK(h, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond{};
    if (si || !h->use_loop) CK(h, cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault));
    KParams<R> plain = make_params<R>(h, 0, 0);
    KParams<R> loop = make_params<R>(h, 1, cond);
    void *a_plain[] = {&plain};
    void *a_loop[] = {&loop};
    int n_mat = (int)h->mats.size();
    void *a_march[] = {&plain, &n_mat};
    IterState *st = h->d_st;
    void *a_st[] = {&st};
    cudaGraphNode_t n_begin, n_prev, n_while, n_commit;
    int rc = add_kernel(h, g, &n_begin, nullptr, 0, (const void *)&ocik::k_step_begin, dim3(1), dim3(1), a_st);
    if (rc) return rc;
    n_prev = n_begin;
    if (!si && h->use_loop && h->use_async && !bar_loop) {
        // barrier-free loop: zero its sync block, one cooperative launch that
        // iterates and ends the step
        cudaMemsetParams mp{};
        mp.dst = h->as;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = h->as_zero_bytes / 4;
        mp.height = 1;
        cudaGraphNode_t n_zero, n_loop;
        CK(h, cudaGraphAddMemsetNode(&n_zero, g, &n_prev, 1, &mp));
        rc = add_kernel(h, g, &n_loop, &n_zero, 1, h->cells_async, dim3(h->cells_grid), dim3(h->cells_block), a_plain,
                        h->cells_smem);
        if (rc) return rc;
        cudaLaunchAttributeValue v{};
        v.cooperative = 1;
        CK(h, cudaGraphKernelNodeSetAttribute(n_loop, cudaLaunchAttributeCooperative, &v));
        CK(h, cudaGraphInstantiate(eout, g, 0));
        *gout = g;
        return OCI_OK;
    }
    if (!si && h->use_loop) {
        // the persistent loop ends the step itself (commit in the same launch)
        cudaGraphNode_t n_loop;
        KParams<R> lc = plain;
        lc.loop_commit = 1;
        void *a_lc[] = {&lc};
        rc = add_loop(h, g, &n_prev, &n_loop, a_lc);
        if (rc) return rc;
        CK(h, cudaGraphInstantiate(eout, g, 0));
        *gout = g;
        return OCI_OK;
    }
    if (si) {
        cudaGraphNode_t n_prep;
        rc = add_kernel(h, g, &n_prep, &n_prev, 1, h->ks.si_prep, dim3(h->grid_pc), dim3(kBlock), a_plain);
        if (rc) return rc;
        n_prev = n_prep;
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CK(h, cudaGraphAddNode(&n_while, g, &n_prev, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphNode_t b_cells;
    // parallel-prefix sweep operands (used when h->sweep == OCI_SWEEP_SCAN)
    int nseg = h->scan_nseg;
    const int nch = 2 * h->P;
    ocik::Aff<R> *agg = (ocik::Aff<R> *)h->scan_mem;
    r2<R> *enter = h->scan_mem ? (r2<R> *)((char *)h->scan_mem + (((size_t)nch * nseg * sizeof(ocik::Aff<R>) + 255) &
                                                                 ~(size_t)255))
                               : nullptr;
    void *a_red[] = {&plain, &agg};
    void *a_seg[] = {&plain, &agg, &enter, &nseg};
    void *a_app[] = {&plain, &enter};
    if (si && h->sweep == OCI_SWEEP_SCAN) {
        cudaGraphNode_t b_red, b_seg, b_app;
        rc = add_kernel(h, body, &b_red, nullptr, 0, h->ks.scan_reduce, dim3(nseg, nch), dim3(ocik::SCAN_T), a_red);
        if (!rc) rc = add_kernel(h, body, &b_seg, &b_red, 1, h->ks.scan_segments, dim3(h->P), dim3(32), a_seg);
        if (!rc) rc = add_kernel(h, body, &b_app, &b_seg, 1, h->ks.scan_apply, dim3(nseg, nch), dim3(ocik::SCAN_T), a_app);
        if (rc) return rc;
        rc = add_kernel(h, body, &b_cells, &b_app, 1, h->cells_si, dim3(h->cells_grid), dim3(h->cells_block), a_loop,
                        h->cells_smem);
    } else if (si) {
        cudaGraphNode_t b_march;
        const int nm = h->bcl == OCI_BC_REFLECT ? h->P : 2 * h->P;
        rc = add_kernel(h, body, &b_march, nullptr, 0, h->ks.march, dim3(nm), dim3(32), a_march);
        if (rc) return rc;
        rc = add_kernel(h, body, &b_cells, &b_march, 1, h->cells_si, dim3(h->cells_grid), dim3(h->cells_block),
                        a_loop, h->cells_smem);
    } else {
        rc = add_iterations(h, body, h->cells_oci, a_loop);
    }
    if (rc) return rc;
    rc = add_kernel(h, g, &n_commit, &n_while, 1, si ? h->ks.commit_si : h->ks.commit_oci, dim3(h->grid_pc),
                    dim3(kBlock), a_plain);
    if (rc) return rc;
    CK(h, cudaGraphInstantiate(eout, g, 0));
    *gout = g;
    return OCI_OK;
}

// Continuation of a paused OCI step: WHILE { cells } -> commit (or the
// persistent loop, which commits in the same launch).
template <typename R>
int build_cont_graph(oci_handle *h)
{
    cudaGraph_t g;
    CK(h, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond{};
    if (!h->use_loop) CK(h, cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault));
    KParams<R> plain = make_params<R>(h, 0, 0);
    KParams<R> loop = make_params<R>(h, 1, cond);
    void *a_plain[] = {&plain};
    void *a_loop[] = {&loop};
    if (h->use_loop) {
        cudaGraphNode_t n_loop;
        KParams<R> lc = plain;
        lc.loop_commit = 1;
        void *a_lc[] = {&lc};
        int rc = add_loop(h, g, nullptr, &n_loop, a_lc);
        if (rc) return rc;
        CK(h, cudaGraphInstantiate(&h->exec_cont, g, 0));
        h->graph_cont = g;
        return OCI_OK;
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t n_while, n_commit;
    CK(h, cudaGraphAddNode(&n_while, g, nullptr, nullptr, 0, &cp));
    int rc = add_iterations(h, cp.conditional.phGraph_out[0], h->cells_oci, a_loop);
    if (rc) return rc;
    rc = add_kernel(h, g, &n_commit, &n_while, 1, h->ks.commit_oci, dim3(h->grid_pc), dim3(kBlock), a_plain);
    if (rc) return rc;
    CK(h, cudaGraphInstantiate(&h->exec_cont, g, 0));
    h->graph_cont = g;
    return OCI_OK;
}

// Correction iteration of a stalled FP32 step: WHILE { cells_lin } -> commit_lin.
int build_lin_graph(oci_handle *h)
{
    cudaGraph_t g;
    CK(h, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    CK(h, cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault));
    KParams<float> plain = make_params<float>(h, 0, 0);
    KParams<float> loop = make_params<float>(h, 1, cond);
    void *a_plain[] = {&plain};
    void *a_loop[] = {&loop};
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t n_while, n_commit, b_cells;
    CK(h, cudaGraphAddNode(&n_while, g, nullptr, nullptr, 0, &cp));
    int rc = add_kernel(h, cp.conditional.phGraph_out[0], &b_cells, nullptr, 0, h->cells_lin, dim3(h->cells_grid),
                        dim3(h->cells_block), a_loop, h->cells_smem);
    if (rc) return rc;
    rc = add_kernel(h, g, &n_commit, &n_while, 1, h->ks.commit_lin, dim3(h->grid_pc), dim3(kBlock), a_plain);
    if (rc) return rc;
    CK(h, cudaGraphInstantiate(&h->exec_lin, g, 0));
    h->graph_lin = g;
    return OCI_OK;
}

// OCI step with the BF16 halo: begin -> entry iteration (float faces in, BF16
// out) -> BF16 persistent loop (until ST_SWITCH) -> exit iteration (BF16 in,
// float out) -> FP32 persistent loop (which commits).  The last iteration always
// reads float faces, so the commit is the plain one.
int build_halo_graph(oci_handle *h)
{
    cudaGraph_t g;
    CK(h, cudaGraphCreate(&g, 0));
    KParams<float> plain = make_params<float>(h, 0, 0);
    void *a_plain[] = {&plain};
    IterState *st = h->d_st;
    void *a_st[] = {&st};
    const dim3 grid(h->cells_grid), block(h->cells_block);
    cudaGraphNode_t n_begin, n_entry, n_hloop, n_exit, n_loop, n_zero;
    int rc = add_kernel(h, g, &n_begin, nullptr, 0, (const void *)&ocik::k_step_begin, dim3(1), dim3(1), a_st);
    if (!rc) rc = add_kernel(h, g, &n_entry, &n_begin, 1, h->hk.entry, grid, block, a_plain, h->cells_smem);
    if (rc) return rc;
    cudaMemsetParams mp{};
    mp.dst = h->loop_bar;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned);
    mp.width = 1;
    mp.height = 1;
    CK(h, cudaGraphAddMemsetNode(&n_zero, g, &n_entry, 1, &mp));
    rc = add_kernel(h, g, &n_hloop, &n_zero, 1, h->hk.loop, grid, block, a_plain, h->cells_smem);
    if (rc) return rc;
    cudaLaunchAttributeValue v{};
    v.cooperative = 1;
    CK(h, cudaGraphKernelNodeSetAttribute(n_hloop, cudaLaunchAttributeCooperative, &v));
    KParams<float> lc = plain;
    lc.loop_commit = 1;
    void *a_lc[] = {&lc};
    rc = add_kernel(h, g, &n_exit, &n_hloop, 1, h->hk.exit, grid, block, a_plain, h->cells_smem);
    if (!rc) rc = add_loop(h, g, &n_exit, &n_loop, a_lc);
    if (rc) return rc;
    CK(h, cudaGraphInstantiate(&h->exec_oci_h, g, 0));
    h->graph_oci_h = g;
    return OCI_OK;
}

// BF16 face buffers: zeroed, with the prescribed boundary data (faceP[.][0],
// faceM[.][J]) of the float buffers rounded into both.
__global__ void k_halo_bounds(const r2<float> *fP0, const r2<float> *fMJ, int P, unsigned *hP0, unsigned *hP1,
                              unsigned *hMJ0, unsigned *hMJ1)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const unsigned a = ocik::pack_bf16x2(fP0[i].x, fP0[i].y), b = ocik::pack_bf16x2(fMJ[i].x, fMJ[i].y);
        hP0[i] = a;
        hP1[i] = a;
        hMJ0[i] = b;
        hMJ1[i] = b;
    }
}

int halo_setup(oci_handle *h)
{
    // the BF16 kernels are instantiated for 8-row chunks and a 2-stage ring only
    if (h->prec != OCI_FP32 || !h->use_loop || h->P % 4 != 0 || h->ks.tma_chunk != 8 || h->ks.tma_stages != 2 ||
        !ocik::kernel_set_bf16(h->lpc, h->ppl, &h->hk))
        return OCI_EINVAL;
    int sms = 0, per_sm = 0;
    for (const void *fn : {h->hk.entry, h->hk.loop, h->hk.exit})
        CK(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->cells_smem));
    CK(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, h->hk.loop, h->cells_block, h->cells_smem));
    if (h->cells_grid > sms * per_sm) return OCI_EINVAL;  // the cooperative loop would not fit
    const size_t fb = (size_t)(h->J + 1) * h->P * 4, fa = (fb + 255) & ~(size_t)255;
    if (!h->hface_mem && cudaMalloc(&h->hface_mem, 4 * fa) != cudaSuccess) return OCI_ENOMEM;
    char *b = (char *)h->hface_mem;
    h->hfP[0] = (unsigned *)b;
    h->hfP[1] = (unsigned *)(b + fa);
    h->hfM[0] = (unsigned *)(b + 2 * fa);
    h->hfM[1] = (unsigned *)(b + 3 * fa);
    CK(h, cudaMemsetAsync(h->hface_mem, 0, 4 * fa, h->stream));
    const size_t JP = (size_t)h->J * h->P;
    k_halo_bounds<<<1, 256, 0, h->stream>>>((const r2<float> *)h->faceP[0], (const r2<float> *)h->faceM[0] + JP, h->P,
                                             h->hfP[0], h->hfP[1], h->hfM[0] + JP, h->hfM[1] + JP);
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->stream));
    return build_halo_graph(h);
}

int ensure_graphs(oci_handle *h)
{
    if (h->exec_oci && !h->exec_si) {
        return h->prec == OCI_FP64 ? build_graph<double>(h, true, &h->graph_si, &h->exec_si)
                                   : build_graph<float>(h, true, &h->graph_si, &h->exec_si);
    }
    if (h->exec_oci) return OCI_OK;
    int rc = h->prec == OCI_FP64 ? build_graph<double>(h, false, &h->graph_oci, &h->exec_oci)
                                 : build_graph<float>(h, false, &h->graph_oci, &h->exec_oci);
    if (rc && h->use_loop) {
        // a cooperative kernel node was refused: iterate with one launch per iteration
        (void)cudaGetLastError();
        h->use_loop = false;
        h->use_async = false;
        rc = h->prec == OCI_FP64 ? build_graph<double>(h, false, &h->graph_oci, &h->exec_oci)
                                 : build_graph<float>(h, false, &h->graph_oci, &h->exec_oci);
    }
    if (rc && h->pdl_graph && h->staged) {
        // programmatic edges refused inside the loop body: plain single launches
        (void)cudaGetLastError();
        if (h->graph_oci) cudaGraphDestroy(h->graph_oci);
        h->graph_oci = nullptr;
        h->exec_oci = nullptr;
        h->pdl_graph = false;
        rc = h->prec == OCI_FP64 ? build_graph<double>(h, false, &h->graph_oci, &h->exec_oci)
                                 : build_graph<float>(h, false, &h->graph_oci, &h->exec_oci);
    }
    if (!rc) rc = h->prec == OCI_FP64 ? build_graph<double>(h, true, &h->graph_si, &h->exec_si)
                                      : build_graph<float>(h, true, &h->graph_si, &h->exec_si);
    return rc;
}

int launch_lift(oci_handle *h, const void *fn)
{
    if (h->prec == OCI_FP64) {
        KParams<double> p = make_params<double>(h, 0, 0);
        void *a[] = {&p, &h->nn_phat, &h->nn_hist[0], &h->nn_hist[1]};
        CK(h, cudaLaunchKernel(fn, dim3(h->grid_pc), dim3(kBlock), a, 0, h->stream));
    } else {
        KParams<float> p = make_params<float>(h, 0, 0);
        void *a[] = {&p, &h->nn_phat, &h->nn_hist[0], &h->nn_hist[1]};
        CK(h, cudaLaunchKernel(fn, dim3(h->grid_pc), dim3(kBlock), a, 0, h->stream));
    }
    return OCI_OK;
}

int launch_guess(oci_handle *h)
{
    if (h->prec == OCI_FP64) {
        KParams<double> p = make_params<double>(h, 0, 0);
        void *a[] = {&p};
        CK(h, cudaLaunchKernel(h->ks.guess, dim3(h->grid_pc), dim3(kBlock), a, 0, h->stream));
    } else {
        KParams<float> p = make_params<float>(h, 0, 0);
        void *a[] = {&p};
        CK(h, cudaLaunchKernel(h->ks.guess, dim3(h->grid_pc), dim3(kBlock), a, 0, h->stream));
    }
    return OCI_OK;
}

// Make the device's iteration controls equal to c (copied only when they differ).
int set_device_cfg(oci_handle *h, const IterConfig &c)
{
    if (std::memcmp(&c, &h->cfg_dev, sizeof(IterConfig)) == 0) return OCI_OK;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(h->d_cfg, &c, sizeof(IterConfig), cudaMemcpyHostToDevice));
    h->cfg_dev = c;
    return OCI_OK;
}

int upload_cfg(oci_handle *h) { return set_device_cfg(h, h->cfg); }

int read_state(oci_handle *h, IterState *s)
{
    CK(h, cudaMemcpyAsync(h->h_st, h->d_st, sizeof(IterState), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *s = *h->h_st;
    return OCI_OK;
}

size_t face_bytes(const oci_handle *h) { return (size_t)(h->J + 1) * h->P * 2 * rsize(h); }

// Save / restore the iterate the next iteration will read (both face arrays
// and the scalar-flux moments) for the corrector's safeguard.
int corr_copy(oci_handle *h, const IterState &s, bool save)
{
    const int fb = (s.base + s.iter) & 1;
    const size_t fbytes = face_bytes(h);
    char *bak = (char *)h->nn_face_bak;
    void *ph = h->phi[s.iter & 1];
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    if (save) {
        CK(h, cudaMemcpyAsync(bak, h->faceP[fb], fbytes, k, h->stream));
        CK(h, cudaMemcpyAsync(bak + fbytes, h->faceM[fb], fbytes, k, h->stream));
        CK(h, cudaMemcpyAsync(h->nn_phi_bak, ph, (size_t)h->J * 32, k, h->stream));
    } else {
        CK(h, cudaMemcpyAsync(h->faceP[fb], bak, fbytes, k, h->stream));
        CK(h, cudaMemcpyAsync(h->faceM[fb], bak + fbytes, fbytes, k, h->stream));
        CK(h, cudaMemcpyAsync(ph, h->nn_phi_bak, (size_t)h->J * 32, k, h->stream));
    }
    return OCI_OK;
}

// phat = network(phi_{n-1}, phi_{n-2}, static inputs), then lift into the guess.
int nn_guess(oci_handle *h)
{
    cudaStream_t s = h->stream;
    if (oci_nn_features(h->nn_hist[0], h->nn_hist[1], h->nn_stat, h->nn_qfeat, 1, h->J, h->nn_in, h->nn_scale, s) ||
        oci_nn_forward(h->nn_params, h->nn_in, 1, h->J, h->nn_out, h->nn_ws, h->nn_ws_bytes, s) ||
        oci_nn_predict(h->nn_hist[0], h->nn_out, h->nn_scale, 1, h->J, h->nn_phat, s))
        return cuda_fail(h, cudaGetLastError(), "network inference");
    return launch_lift(h, h->ks.lift_guess);
}

// A stalled FP32 step: save the halo h0, evaluate r0 = G(h0) - h0 and phi(h0)
// in FP64, iterate d = B d + r0 from d = 0 in FP32, commit h0 + d.
int refine_step(oci_handle *h, IterState *s)
{
    if (!h->exec_lin) {
        int rc = build_lin_graph(h);
        if (rc) return rc;
    }
    // the latest iterate: rotated through three buffers by the barrier-free loop
    const int fb = s->rot3 ? s->cur_face : (s->base + s->iter) & 1;
    const size_t fbytes = face_bytes(h);
    CK(h, cudaMemcpyAsync(h->ref_h0P, h->faceP[fb], fbytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->ref_h0M, h->faceM[fb], fbytes, cudaMemcpyDeviceToDevice, h->stream));
    KParams<float> p = make_params<float>(h, 0, 0);
    ocik::RefineArgs q{h->ref_tab, h->ref_par, h->ref_muw, (r4<float> *)h->ref_r0, (float2 *)h->ref_phi};
    void *a[] = {&p, &q};
    CK(h, cudaLaunchKernel(h->ks.refine, dim3(h->grid_pc), dim3(kBlock), a, 0, h->stream));
    IterState *st = h->d_st;
    void *a_st[] = {&st};
    CK(h, cudaLaunchKernel((const void *)&ocik::k_refine_setup, dim3(1), dim3(1), a_st, 0, h->stream));
    // the correction starts from d = 0 and phi_lin = 0 and has homogeneous
    // boundary data: clear both face buffers (boundary slots included; h0 is saved)
    for (int b = 0; b < 2; ++b) {
        CK(h, cudaMemsetAsync(h->faceP[b], 0, fbytes, h->stream));
        CK(h, cudaMemsetAsync(h->faceM[b], 0, fbytes, h->stream));
    }
    CK(h, cudaMemsetAsync(h->phi[(s->iter + 1) & 1], 0, (size_t)h->J * 32, h->stream));
    CK(h, cudaGraphLaunch(h->exec_lin, h->stream));
    int rc = read_state(h, s);
    if (rc) return rc;
    ++h->refinements;
    // boundary data slots of both face buffers (zeroed for the correction)
    return upload_boundaries(h, h->bc_left_host.empty() ? nullptr : h->bc_left_host.data(),
                             h->bc_right_host.empty() ? nullptr : h->bc_right_host.data());
}

// Per-material inverses, cells grouped by material, cuBLAS handle.
int dense_setup(oci_handle *h)
{
    const int J = h->J, P = h->P, nm = (int)h->mats.size(), n = 8 * P;
    const size_t rs = rsize(h);
    const size_t inv_bytes = (size_t)nm * n * n * rs, col_bytes = (size_t)J * n * rs;
    if (inv_bytes > ((size_t)4 << 30) || col_bytes > ((size_t)16 << 30)) return OCI_EINVAL;
    std::vector<double> mu_p(P), w_p(P), inv, all;
    for (int p = 0; p < P; ++p) { mu_p[p] = h->mu[P + p]; w_p[p] = h->w[P + p]; }
    all.reserve((size_t)nm * n * n);
    for (int m = 0; m < nm; ++m) {
        const Material &mt = h->mats[m];
        const double e = std::isinf(h->v) ? 0.0 : mt.dx / (2.0 * h->v * h->dt);
        if (!ocik::dense_inverse(mu_p.data(), w_p.data(), P, mt.dx, mt.st, mt.ss, e, inv)) return OCI_EINVAL;
        all.insert(all.end(), inv.begin(), inv.end());
    }
    std::vector<int> perm(J), off(nm + 1, 0);
    for (int j = 0; j < J; ++j) ++off[h->mat[j] + 1];
    for (int m = 0; m < nm; ++m) off[m + 1] += off[m];
    {
        std::vector<int> next(off.begin(), off.end() - 1);
        for (int j = 0; j < J; ++j) perm[next[h->mat[j]]++] = j;
    }
    ocik::DenseBuffers &d = h->dense;
    const size_t a0 = (inv_bytes + 255) & ~(size_t)255, a1 = (col_bytes + 255) & ~(size_t)255;
    if (cudaMalloc(&d.mem, a0 + 2 * a1 + (size_t)J * 4) != cudaSuccess) {
        d.mem = nullptr;
        return OCI_ENOMEM;
    }
    char *b = (char *)d.mem;
    d.minv = b;
    d.C = b + a0;
    d.Psi = b + a0 + a1;
    d.perm = (int *)(b + a0 + 2 * a1);
    d.ncols = J;
    d.col_off = off;
    int rc = upload_real(h, d.minv, all);
    if (rc) return rc;
    CK(h, cudaMemcpy(d.perm, perm.data(), sizeof(int) * J, cudaMemcpyHostToDevice));
    if (ocik::dense_blas_create(&d.blas)) return cuda_fail(h, cudaErrorUnknown, "cublasCreate");
    h->dense_grid = std::max(1, std::min((J + 7) / 8, h->grid_cells));
    return OCI_OK;
}

void dense_free(oci_handle *h)
{
    ocik::dense_blas_destroy(h->dense.blas);
    if (h->dense.mem) cudaFree(h->dense.mem);
    h->dense = ocik::DenseBuffers{};
}

int dense_iterate(oci_handle *h)
{
    int rc;
    if (h->prec == OCI_FP64) rc = ocik::dense_iteration(make_params<double>(h, 0, 0), h->dense, h->dense_grid, h->stream);
    else rc = ocik::dense_iteration(make_params<float>(h, 0, 0), h->dense, h->dense_grid, h->stream);
    return rc ? cuda_fail(h, cudaGetLastError(), "dense iteration") : OCI_OK;
}

// One OCI step with the dense inverse: the loop runs on the host (one status
// read per iteration), then the shared commit kernel.
int dense_step(oci_handle *h, IterState *s)
{
    IterConfig c = h->cfg;
    c.stall_floor = 0.0;  // no FP32 refinement on this path
    c.pause_at = -1;
    int rc = set_device_cfg(h, c);
    if (rc) return rc;
    IterState *st = h->d_st;
    void *a_st[] = {&st};
    CK(h, cudaLaunchKernel((const void *)&ocik::k_step_begin, dim3(1), dim3(1), a_st, 0, h->stream));
    for (int it = 0; it < c.max_iter + 2; ++it) {
        if ((rc = dense_iterate(h)) || (rc = read_state(h, s))) return rc;
        if (s->status != ocik::ST_RUNNING) break;
    }
    KParams<double> pd = make_params<double>(h, 0, 0);
    KParams<float> pf = make_params<float>(h, 0, 0);
    void *args[] = {h->prec == OCI_FP64 ? (void *)&pd : (void *)&pf};
    CK(h, cudaLaunchKernel(h->ks.commit_oci, dim3(h->grid_pc), dim3(kBlock), args, 0, h->stream));
    return OCI_OK;
}

// Backward-Euler tables: 1/t per material and pair, t = a - i mu/2,
// a = (mu + dx Sigma)/2 + dx/(2 v dt); scalar capacitance K = 1/(1 - s m),
// m = sum_p 2 w_p Re(1/t).
int be_setup(oci_handle *h)
{
    const int P = h->P, nm = (int)h->mats.size();
    std::vector<double> tab((size_t)nm * P * 2), K(nm);
    for (int m = 0; m < nm; ++m) {
        const Material &mt = h->mats[m];
        const double e = std::isinf(h->v) ? 0.0 : mt.dx / (2.0 * h->v * h->dt);
        const double s = mt.dx * mt.ss / 4.0;
        double msum = 0.0;
        for (int p = 0; p < P; ++p) {
            const double mu = h->mu[P + p];
            const std::complex<double> it = 1.0 / std::complex<double>((mu + mt.dx * mt.st) / 2.0 + e, -mu / 2.0);
            tab[((size_t)m * P + p) * 2] = it.real();
            tab[((size_t)m * P + p) * 2 + 1] = it.imag();
            msum += 2.0 * h->w[P + p] * it.real();
        }
        const double den = 1.0 - s * msum;
        if (!(std::fabs(den) > 0.0) || !std::isfinite(den)) return OCI_EINVAL;
        K[m] = 1.0 / den;
    }
    const size_t rs = rsize(h), tb = ((size_t)nm * P * 2 * rs + 255) & ~(size_t)255;
    const size_t kb = ((size_t)nm * 8 + 255) & ~(size_t)255;
    if (cudaMalloc(&h->be_mem, tb + kb + (size_t)nm * 8) != cudaSuccess) {
        h->be_mem = nullptr;
        return OCI_ENOMEM;
    }
    h->be_tab = h->be_mem;
    h->be_K = (double *)((char *)h->be_mem + tb);
    h->be_Kf = (float2 *)((char *)h->be_mem + tb + kb);
    std::vector<float> kf((size_t)nm * 2);
    for (int m = 0; m < nm; ++m) {
        kf[2 * m] = (float)K[m];
        kf[2 * m + 1] = (float)(K[m] - (double)kf[2 * m]);
    }
    int rc = upload_real(h, h->be_tab, tab);
    if (rc) return rc;
    CK(h, cudaMemcpy(h->be_K, K.data(), sizeof(double) * nm, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->be_Kf, kf.data(), sizeof(float) * kf.size(), cudaMemcpyHostToDevice));
    return OCI_OK;
}

// BE step graph: begin -> WHILE { be_cells } -> be_commit.
template <typename R>
int build_be_graph(oci_handle *h)
{
    cudaGraph_t g;
    CK(h, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    CK(h, cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault));
    KParams<R> plain = make_params<R>(h, 0, 0);
    KParams<R> loop = make_params<R>(h, 1, cond);
    ocik::BeArgs<R> be{(const r2<R> *)h->be_tab, h->be_K, h->be_Kf};
    void *a_plain[] = {&plain, &be};
    void *a_loop[] = {&loop, &be};
    IterState *st = h->d_st;
    void *a_st[] = {&st};
    const int grid = std::max(1, std::min((h->J + 7) / 8, h->grid_cells));
    cudaGraphNode_t n_begin, n_while, n_commit, b_cells;
    int rc = add_kernel(h, g, &n_begin, nullptr, 0, (const void *)&ocik::k_step_begin, dim3(1), dim3(1), a_st);
    if (rc) return rc;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CK(h, cudaGraphAddNode(&n_while, g, &n_begin, nullptr, 1, &cp));
    rc = add_kernel(h, cp.conditional.phGraph_out[0], &b_cells, nullptr, 0, h->ks.be_cells, dim3(grid), dim3(kBlock),
                    a_loop);
    if (!rc) rc = add_kernel(h, g, &n_commit, &n_while, 1, h->ks.be_commit, dim3(grid), dim3(kBlock), a_plain);
    if (rc) return rc;
    CK(h, cudaGraphInstantiate(&h->exec_be, g, 0));
    h->graph_be = g;
    return OCI_OK;
}

int map_status(int s)
{
    switch (s) {
    case ocik::ST_CONVERGED: return OCI_OK;
    case ocik::ST_MAXITER: return OCI_ENOTCONV;
    case ocik::ST_NAN: return OCI_ENAN;
    case ocik::ST_STALL: return OCI_ENOTCONV;
    case ocik::ST_HELD: return OCI_ESKIPPED;
    default: return OCI_ETIMEOUT;
    }
}

// NVTX range around one time step (visible in Nsight timelines; no cost without a tool).
struct StepRange {
    explicit StepRange(const char *name) { nvtxRangePushA(name); }
    ~StepRange() { nvtxRangePop(); }
};

// Domain decomposition: the cut faces of the iterate the next iteration reads
// (face buffer (base + iter) & 1, read on the device).  Export: the outgoing
// -mu flux at face 0 and +mu flux at face J (written by cells 0 and J-1);
// import: the incident +mu flux at face 0 and -mu flux at face J (the boundary
// slots, which no cell writes).  [P] r2 (k, k+1/2) per pair; NULL skips a side.
template <typename R>
__global__ void k_dd_faces(const IterState *st, r2<R> *fP0, r2<R> *fP1, r2<R> *fM0, r2<R> *fM1, int J, int P,
                           r2<R> *left, r2<R> *right, int import)
{
    const int b = (st->base + st->iter) & 1;
    r2<R> *fP = b ? fP1 : fP0, *fM = b ? fM1 : fM0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        if (import) {
            if (left) fP[i] = left[i];
            if (right) fM[(size_t)J * P + i] = right[i];
        } else {
            if (left) left[i] = fM[i];
            if (right) right[i] = fP[(size_t)J * P + i];
        }
    }
}

// Domain decomposition: the step's decision taken from the global sums.
__global__ void k_dd_decide(IterState *st, int status, double resid, double d2, double p2)
{
    st->status = status;
    st->resid = resid;
    st->d2 = d2;
    st->p2 = p2;
}

int dd_faces(oci_handle *h, void *left, void *right, int import)
{
    const int grid = (h->P + 255) / 256;
    if (h->prec == OCI_FP64)
        k_dd_faces<double><<<grid, 256, 0, h->stream>>>(h->d_st, (r2<double> *)h->faceP[0], (r2<double> *)h->faceP[1],
                                                        (r2<double> *)h->faceM[0], (r2<double> *)h->faceM[1], h->J,
                                                        h->P, (r2<double> *)left, (r2<double> *)right, import);
    else
        k_dd_faces<float><<<grid, 256, 0, h->stream>>>(h->d_st, (r2<float> *)h->faceP[0], (r2<float> *)h->faceP[1],
                                                       (r2<float> *)h->faceM[0], (r2<float> *)h->faceM[1], h->J, h->P,
                                                       (r2<float> *)left, (r2<float> *)right, import);
    CK(h, cudaGetLastError());
    return OCI_OK;
}

// One OCI iteration as a single launch (no graph, no local decision: the
// device controls of a decomposed step never end it).
int dd_iteration(oci_handle *h)
{
    KParams<double> pd = make_params<double>(h, 0, 0);
    KParams<float> pf = make_params<float>(h, 0, 0);
    void *args[] = {h->prec == OCI_FP64 ? (void *)&pd : (void *)&pf};
    CK(h, cudaLaunchKernel(h->cells_oci, dim3(h->cells_grid), dim3(h->cells_block), args, h->cells_smem, h->stream));
    return OCI_OK;
}

int run_step(oci_handle *h, bool si, oci_stats *st)
{
    if (!h) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    const StepRange range(si ? "si_step" : (h->scheme == OCI_TIME_BE ? "oci_step (backward Euler)" : "oci_step"));
    CK(h, cudaSetDevice(h->device));
    int rc = ensure_graphs(h);
    if (!rc) rc = apply_pending_source(h);
    if (rc) return rc;
    int launches = 0;  // kernels of this library enqueued for the step
    if (!h->guess_valid) {
        rc = launch_guess(h);
        if (rc) return rc;
        ++launches;
    }
    bool nn = !si && h->nn_mode != OCI_NN_OFF && h->scheme == OCI_TIME_MB;
    int trial_slot = -1;  // adaptive mode: 0 plain / 1 guessed step of a trial, 2 plain lead-in step
    if (nn && h->nn_mode == OCI_NN_GUESS_ADAPTIVE) {
        if (h->nn_trial < 0) {
            trial_slot = 2;
            nn = false;
        } else if (h->nn_trial < 4) {
            trial_slot = (h->nn_trial == 1 || h->nn_trial == 2) ? 1 : 0;
            nn = trial_slot == 1;
        } else {
            nn = h->nn_use;
        }
    }
    int accepts = 0, rejects = 0;
    const int unroll = (h->staged && h->pdl_graph) ? kUnroll : 1;  // iteration launches per WHILE body
    auto body_launches = [&](int iters) { return unroll * ((iters + unroll - 1) / unroll); };
    int corrections = 0, graph_runs = 0;
    bool halo_graph = false, async_run = false;
    CK(h, cudaEventRecord(h->ev0, h->stream));
    if (nn) {
        rc = nn_guess(h);
        if (rc) return rc;
        h->guess_valid = false;
        ++accepts;
        launches += 10;  // scale, features, weight rounding, 5 layers, predict, lift
    }
    IterState s{};
    if (h->scheme == OCI_TIME_BE) {
        if (si) return OCI_EINVAL;
        if (!h->exec_be) {
            rc = h->prec == OCI_FP64 ? build_be_graph<double>(h) : build_be_graph<float>(h);
            if (rc) return rc;
        }
        IterConfig c = h->cfg;
        c.stall_floor = 0.0;
        c.pause_at = -1;
        if ((rc = set_device_cfg(h, c))) return rc;
        CK(h, cudaGraphLaunch(h->exec_be, h->stream));
        ++graph_runs;
    } else if (!si && h->solver == OCI_SOLVER_DENSE) {
        if ((rc = dense_step(h, &s))) return rc;
    } else if (nn && h->nn_mode == OCI_NN_GUESS_CORRECT) {
        if (!h->exec_cont) {
            rc = h->prec == OCI_FP64 ? build_cont_graph<double>(h) : build_cont_graph<float>(h);
            if (rc) return rc;
        }
        const int k = h->nn_kcorr, m_check = std::min(h->nn_kcorr, 8);
        bool correcting = true;
        h->cfg.pause_at = k;
        if ((rc = upload_cfg(h))) return rc;
        // pauses need the barrier loop (its iterate stays in the two-buffer order)
        if (h->use_async && !h->exec_oci_bar) {
            rc = build_graph<float>(h, false, &h->graph_oci_bar, &h->exec_oci_bar, true);
            if (rc) return rc;
        }
        CK(h, cudaGraphLaunch(h->use_async ? h->exec_oci_bar : h->exec_oci, h->stream));
        ++graph_runs;
        for (;;) {
            if ((rc = read_state(h, &s))) return rc;
            if (s.status != ocik::ST_RUNNING) break;
            if (correcting) {
                // pause: try a correction toward phat, keep it only if it helped
                const double before = s.resid;
                if ((rc = corr_copy(h, s, true)) || (rc = launch_lift(h, h->ks.lift_corr))) return rc;
                ++corrections;
                h->cfg.pause_at = s.iter + m_check;
                if ((rc = upload_cfg(h))) return rc;
                CK(h, cudaGraphLaunch(h->exec_cont, h->stream));
                ++graph_runs;
                IterState s2{};
                if ((rc = read_state(h, &s2))) return rc;
                if (s2.status != ocik::ST_RUNNING) { s = s2; ++accepts; break; }
                if (s2.resid > before) {
                    if ((rc = corr_copy(h, s2, false))) return rc;  // back to the saved iterate
                    ++rejects;
                    correcting = false;
                } else {
                    ++accepts;
                }
                s = s2;
            }
            h->cfg.pause_at = correcting ? s.iter + k : -1;
            if ((rc = upload_cfg(h))) return rc;
            CK(h, cudaGraphLaunch(h->exec_cont, h->stream));
            ++graph_runs;
        }
        h->cfg.pause_at = -1;
        if ((rc = upload_cfg(h))) return rc;
    } else {
        IterConfig c = h->cfg;
        if (si) c.stall_floor = 0.0;  // SI has no refinement: no stall stop
        if ((rc = set_device_cfg(h, c))) return rc;
        // BF16 halo: entry, BF16 loop and exit take at least three iterations
        halo_graph = !si && h->halo == OCI_HALO_BF16 && h->exec_oci_h && h->cfg.max_iter >= 4;
        async_run = !si && !halo_graph && h->use_async;
        CK(h, cudaGraphLaunch(halo_graph ? h->exec_oci_h : (si ? h->exec_si : h->exec_oci), h->stream));
        ++graph_runs;
    }
    CK(h, cudaEventRecord(h->ev1, h->stream));
    if ((rc = read_state(h, &s))) return rc;  // the step's one synchronisation in the common case
    const int main_iters = s.iter;
    if (h->scheme == OCI_TIME_BE) launches += 2 + main_iters;  // begin, iterations, commit
    else if (!si && h->solver == OCI_SOLVER_DENSE) launches += 2 + 2 * main_iters;  // begin, rhs + out per iteration, commit
    else if (si) launches += 3 + main_iters * (h->sweep == OCI_SWEEP_SCAN ? 4 : 2);  // begin, prep, sweep + cells, commit
    else if (halo_graph) launches += 6;  // begin, entry, BF16 loop, exit, loop, commit
    else if (async_run) launches += 2;   // begin, the barrier-free loop (which ends the step)
    else if (h->use_loop) launches += 1 + graph_runs + corrections;  // begin, one loop (which commits) per graph run, lifts
    else launches += 2 + body_launches(main_iters) + corrections * (unroll + 1);  // begin, bodies, commit, lifts
    int refined = 0;
    if (s.status == ocik::ST_STALL && !si && h->scheme == OCI_TIME_MB && h->cells_lin && h->ks.refine) {
        if ((rc = refine_step(h, &s))) return rc;
        refined = 1;
        launches += 2 + (s.iter - main_iters);  // residual pass, setup, correction iterations, commit
        CK(h, cudaEventRecord(h->ev1, h->stream));
        if ((rc = read_state(h, &s))) return rc;
    }
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->guess_valid = s.committed != 0;
    if (s.committed && h->nn_mem) {
        // history of committed moments for the network: hist[1] <- hist[0] <- phi_out
        std::swap(h->nn_hist[0], h->nn_hist[1]);
        CK(h, cudaMemcpyAsync(h->nn_hist[0], h->phi_out, (size_t)h->J * 32, cudaMemcpyDeviceToDevice, h->stream));
    }
    if (trial_slot >= 0 && s.committed) {
        if (trial_slot < 2) (trial_slot ? h->nn_trial_nn : h->nn_trial_plain) += s.iter;
        if (++h->nn_trial == 4) {
            h->nn_use = h->nn_trial_nn < 0.97 * (double)h->nn_trial_plain;
            h->nn_since_trial = 0;
        }
    } else if (!si && h->nn_mode == OCI_NN_GUESS_ADAPTIVE && h->nn_trial >= 4 && s.committed &&
               ++h->nn_since_trial >= h->nn_kcorr) {
        h->nn_trial = 0;  // test again
        h->nn_trial_plain = h->nn_trial_nn = 0;
    }
    const int status = map_status(s.status);
    if (st) {
        st->iters = s.iter;
        st->status = status;
        st->residual = s.resid;
        st->seconds = ms * 1e-3;
        st->committed = s.committed;
        st->nn_accepts = accepts;
        st->nn_rejects = rejects;
        st->refined = refined;
        st->launches = launches;
    }
    return status;
}


// ------------------------------------------------------------ oci_run_steps
// Steps that run start to end on the device (the FP32 persistent loop that
// ends the step itself) can be queued two deep: the next step is enqueued
// before the host waits for the previous one.
bool queue_capable(const oci_handle *h)
{
    return h->prec == OCI_FP32 && h->use_loop && !h->use_async && h->solver == OCI_SOLVER_WOODBURY &&
           h->scheme == OCI_TIME_MB && h->nn_mode == OCI_NN_OFF &&
           !(h->halo == OCI_HALO_BF16 && h->exec_oci_h && h->cfg.max_iter >= 4);
}

int rs_setup(oci_handle *h)
{
    if (h->rs_mem) return OCI_OK;
    if (!h->rs_st && cudaMallocHost(&h->rs_st, 2 * sizeof(IterState)) != cudaSuccess) {
        h->rs_st = nullptr;
        return OCI_ENOMEM;
    }
    if (!h->rs_up) CK(h, cudaStreamCreateWithFlags(&h->rs_up, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        if (!h->rs_ev0[k]) CK(h, cudaEventCreate(&h->rs_ev0[k]));
        if (!h->rs_ev1[k]) CK(h, cudaEventCreate(&h->rs_ev1[k]));
        for (cudaEvent_t *e : {&h->rs_done[k], &h->rs_ready[k], &h->rs_free[k]})
            if (!*e) CK(h, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    const size_t qb = ((size_t)h->J * 32 + 255) & ~(size_t)255;
    void *m = nullptr;
    if (cudaMalloc(&m, 2 * qb) != cudaSuccess) return OCI_ENOMEM;
    h->rs_stage[0] = (double *)m;
    h->rs_stage[1] = (double *)((char *)m + qb);
    h->rs_mem = m;
    return OCI_OK;
}

// One queued step on the handle's stream: [the chain flag: hold it unless the
// step before it commits], the step graph (prologue, the loop that ends the
// step), its state to the slot's pinned copy.
int rs_launch(oci_handle *h, int slot, bool chain)
{
    if (chain) CK(h, cudaMemsetAsync(&h->d_st->chain, 1, sizeof(int), h->stream));
    CK(h, cudaEventRecord(h->rs_ev0[slot], h->stream));
    CK(h, cudaGraphLaunch(h->exec_oci, h->stream));
    CK(h, cudaEventRecord(h->rs_ev1[slot], h->stream));
    CK(h, cudaMemcpyAsync(h->rs_st + slot, h->d_st, sizeof(IterState), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaEventRecord(h->rs_done[slot], h->stream));
    return OCI_OK;
}

// The published moments at this point of the stream to host dst: a device
// snapshot on the handle's stream, the host copy on the copy stream (the
// slot's snapshot is reused once its previous host copy is done).
int rs_snapshot(oci_handle *h, int slot, double *dst)
{
    const size_t bytes = (size_t)h->J * 32;
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_d2h[slot], 0));
    CK(h, cudaMemcpyAsync(h->phi_snap[slot], h->phi_out, bytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaEventRecord(h->ev_snap[slot], h->stream));
    CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_snap[slot], 0));
    CK(h, cudaMemcpyAsync(dst, h->phi_snap[slot], bytes, cudaMemcpyDeviceToHost, h->copy_stream));
    CK(h, cudaEventRecord(h->ev_d2h[slot], h->copy_stream));
    return OCI_OK;
}

}  // namespace

extern "C" {

int oci_create(const oci_problem *p, oci_handle **out)
{
    if (!p || !out) return OCI_EINVAL;
    const int J = p->n_cells, N = p->n_ord;
    if (J < 1 || N < 2 || N > 256 || (N & 1)) return OCI_EINVAL;
    if (!p->dx || !p->sigma_t || !p->sigma_s) return OCI_EINVAL;
    if (!(p->v > 0.0) || !(p->dt > 0.0) || !std::isfinite(p->dt)) return OCI_EINVAL;
    if (p->precision != OCI_FP64 && p->precision != OCI_FP32 && p->precision != OCI_FP32_BF16HALO) return OCI_EINVAL;
    if (p->max_iter < 1 || !(p->tol >= 0.0)) return OCI_EINVAL;
    for (int bc : {p->bc_left, p->bc_right})
        if (bc < OCI_BC_VACUUM || bc > OCI_BC_INCIDENT) return OCI_EINVAL;
    if ((p->bc_left == OCI_BC_INCIDENT && !p->psi_bc_left) || (p->bc_right == OCI_BC_INCIDENT && !p->psi_bc_right))
        return OCI_EINVAL;
    for (int j = 0; j < J; ++j) {
        const double dx = p->dx[j], st = p->sigma_t[j], ss = p->sigma_s[j];
        if (!(dx > 0.0) || !std::isfinite(dx) || !(st >= 0.0) || !std::isfinite(st) || !(ss >= 0.0) || ss > st)
            return OCI_EINVAL;
    }
    oci_handle *h = new (std::nothrow) oci_handle();
    if (!h) return OCI_ENOMEM;
    h->J = J;
    h->N = N;
    h->P = N / 2;
    h->prec = p->precision == OCI_FP64 ? OCI_FP64 : OCI_FP32;
    h->bcl = p->bc_left;
    h->bcr = p->bc_right;
    h->v = p->v;
    h->dt = p->dt;
    h->stream = (cudaStream_t)p->cuda_stream;
    h->cfg.max_iter = p->max_iter;
    h->cfg.tol = p->tol;
    h->cfg.commit_unconverged = 0;
    h->cfg.pause_at = -1;
    h->cfg.stall_iters = 8;
    h->cfg.halo_switch = 2e-3;  // BF16 rounding (2^-8 relative) leaves the change near 1e-3
    h->cfg.halo_stall = 2;
    h->cfg.stall_floor = 0.0;  // enabled below for the FP32 path with refinement
    h->cfg.bar_poll_limit = 0;
    h->cfg.bar_shortfall = 0;
    h->cfg.extrap = 0;
    gauss_legendre(N, h->mu, h->w);
    h->dx.assign(p->dx, p->dx + J);
    // materials: distinct (dx, sigma_t, sigma_s)
    std::map<std::tuple<double, double, double>, int> idx;
    h->mat.resize(J);
    for (int j = 0; j < J; ++j) {
        const auto key = std::make_tuple(p->dx[j], p->sigma_t[j], p->sigma_s[j]);
        auto it = idx.find(key);
        if (it == idx.end()) {
            it = idx.emplace(key, (int)h->mats.size()).first;
            h->mats.push_back(Material{p->dx[j], p->sigma_t[j], p->sigma_s[j]});
        }
        h->mat[j] = it->second;
    }
    // kernel layout
    const int P = h->P;
    if (P <= 32) {
        int l = 1;
        while (l < P) l <<= 1;
        h->lpc = l;
        h->ppl = 1;
    } else {
        h->lpc = 32;
        h->ppl = P <= 64 ? 2 : 4;
    }
    const bool okk = h->prec == OCI_FP64 ? ocik::kernel_set_f64(h->lpc, h->ppl, &h->ks)
                                         : ocik::kernel_set_f32(h->lpc, h->ppl, &h->ks);
    if (!okk) { delete h; return OCI_EINVAL; }
    const int warps_per_block = kBlock / 32;
    const int nchunks = (J + h->ks.cells_per_warp - 1) / h->ks.cells_per_warp;
    h->grid_cells = (nchunks + warps_per_block - 1) / warps_per_block;
    const int npc = (J + h->ks.cells_per_warp_pc - 1) / h->ks.cells_per_warp_pc;
    h->grid_pc = (npc + warps_per_block - 1) / warps_per_block;
    if (h->grid_pc > 152 * 16) h->grid_pc = 152 * 16;

    int rc = OCI_OK;
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return OCI_ECUDA; }
    h->cells_oci = h->ks.cells_oci;
    h->cells_si = h->ks.cells_si;
    h->cells_grid = h->grid_cells;
    h->cells_block = kBlock;
    h->cells_smem = 0;
    if (h->ks.cells_oci_tma && P == h->lpc * h->ppl && P >= 2 && std::getenv("OCI_NO_TMA") == nullptr) {
        // staged persistent kernel: as many warps per block as the ring fits in
        // shared memory (<= 8), one block per SM
        int sms = 0, smem_optin = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
            delete h;
            return OCI_ECUDA;
        }
        const unsigned sb = ocik::tma_stage_bytes(h->lpc, h->ks.tma_chunk, P);
        const unsigned per_warp = (unsigned)h->ks.tma_stages * (sb + 8u) + ocik::kXposeBytes;
        int warps = (int)((unsigned)(smem_optin - 2048) / per_warp);
        if (warps > h->ks.tma_max_warps) warps = h->ks.tma_max_warps;
        if (warps >= 1) {
            h->staged = true;
            h->cells_oci = h->ks.cells_oci_tma;
            h->cells_si = h->ks.cells_si_tma;
            h->cells_block = 32 * warps;
            h->cells_smem = ocik::tma_bar_bytes(h->ks.tma_stages, warps) + (unsigned)warps * ocik::kXposeBytes +
                            (unsigned)warps * h->ks.tma_stages * sb;
            // every ring region must start on a 16-byte boundary (bulk copies, vector loads)
            if ((ocik::tma_bar_bytes(h->ks.tma_stages, warps) % 128u) != 0u || (sb % 16u) != 0u ||
                h->cells_smem > (unsigned)smem_optin) {
                delete h;
                return OCI_EINVAL;
            }
            for (const void *fn : {h->cells_oci, h->cells_si})
                if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->cells_smem) !=
                    cudaSuccess) {
                    delete h;
                    return OCI_ECUDA;
                }
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, h->cells_oci, h->cells_block, h->cells_smem) !=
                    cudaSuccess ||
                per_sm < 1) {
                delete h;
                return OCI_ECUDA;
            }
            const int nch = (J + h->ks.cells_per_warp - 1) / h->ks.cells_per_warp;
            const int want = (nch + warps - 1) / warps;
            h->cells_grid = std::min(sms * per_sm, want);
            // persistent loop over the iterations of a step: needs every block
            // resident at once (cooperative launch)
            int coop = 0, per_sm_loop = 0;
            if (h->ks.cells_oci_loop && std::getenv("OCI_NO_LOOP") == nullptr &&
                cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device) == cudaSuccess && coop &&
                cudaFuncSetAttribute(h->ks.cells_oci_loop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)h->cells_smem) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_loop, h->ks.cells_oci_loop, h->cells_block,
                                                              h->cells_smem) == cudaSuccess &&
                h->cells_grid <= sms * per_sm_loop) {
                h->cells_loop = h->ks.cells_oci_loop;
                h->use_loop = true;
                // its barrier-free variant (S_32, S_64, S_128; measured slower than the
                // barrier loop on GB300, so only on request)
                const void *fa = ocik::kernel_async_loop(h->lpc, h->ppl);
                int per_sm_async = 0;
                const char *ea = std::getenv("OCI_ASYNC_LOOP");
                if (fa && h->ks.tma_chunk == 8 && h->ks.tma_stages == 2 && ea && ea[0] == '1' &&
                    cudaFuncSetAttribute(fa, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->cells_smem) ==
                        cudaSuccess &&
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_async, fa, h->cells_block, h->cells_smem) ==
                        cudaSuccess &&
                    h->cells_grid <= sms * per_sm_async) {
                    h->cells_async = fa;
                    h->use_async = true;
                }
            }
            (void)cudaGetLastError();
        }
    }
    // device layout
    const size_t rs = rsize(h), nm = h->mats.size();
    const size_t face = (size_t)(J + 1) * P * 2 * rs;
    size_t sizes[] = {face, face, face, face,                 // faceP[0], faceP[1], faceM[0], faceM[1]
                      (size_t)J * P * 4 * rs,                 // psi_edge
                      (size_t)J * P * 4 * rs,                 // g
                      (size_t)J * 4 * rs,                     // cellq
                      nm * P * 8 * rs,                        // tab
                      nm * 2 * rs,                            // matpar
                      (size_t)P * 2 * rs,                     // muw
                      (size_t)P * 2 * rs,                     // refl
                      (size_t)J * sizeof(int),                // mat
                      nm * sizeof(kmat),                      // matK
                      nm * 32,                                // matKf
                      (size_t)J * 32, (size_t)J * 32, (size_t)J * 32, (size_t)J * 32,  // phi[2], phi0, phi_out
                      (size_t)std::max(h->grid_cells, h->cells_grid) * 16,  // partials
                      sizeof(IterState), sizeof(IterConfig),
                      // refinement (FP32 mode): tab64, par64, muw64, h0P, h0M, r0, phi_ref
                      h->prec == OCI_FP32 ? nm * P * 64 : 0, h->prec == OCI_FP32 ? nm * 16 : 0,
                      h->prec == OCI_FP32 ? (size_t)P * 16 : 0, h->prec == OCI_FP32 ? face : 0,
                      h->prec == OCI_FP32 ? face : 0, h->prec == OCI_FP32 ? (size_t)J * P * 16 : 0,
                      h->prec == OCI_FP32 ? (size_t)J * 32 : 0,
                      // persistent loop: (d2, p2, fault) per block for two iterations, barrier counter
                      (size_t)h->cells_grid * 6 * sizeof(double), sizeof(unsigned),
                      (size_t)J * 32, (size_t)J * 8};                        // q_dev, dx_dev
    const int ns = sizeof(sizes) / sizeof(sizes[0]);
    size_t off[40], total = 0;
    for (int i = 0; i < ns; ++i) {
        off[i] = total;
        // 256 B of slack: staged copies round sizes up to 16 B
        total += (sizes[i] + 256 + 255) & ~(size_t)255;
    }
    if (cudaMalloc(&h->d_base, total) != cudaSuccess) { delete h; return OCI_ENOMEM; }
    h->d_bytes = total;
    char *b = (char *)h->d_base;
    h->faceP[0] = b + off[0]; h->faceP[1] = b + off[1]; h->faceM[0] = b + off[2]; h->faceM[1] = b + off[3];
    h->psi_edge = b + off[4]; h->g = b + off[5]; h->cellq = b + off[6]; h->tab = b + off[7];
    h->matpar = b + off[8]; h->muw = b + off[9]; h->refl = b + off[10]; h->d_mat = (int *)(b + off[11]);
    h->d_matK = (kmat *)(b + off[12]);
    h->d_matKf = b + off[13];
    h->phi[0] = (double *)(b + off[14]); h->phi[1] = (double *)(b + off[15]);
    h->phi0 = (double *)(b + off[16]); h->phi_out = (double *)(b + off[17]);
    h->partials = (double *)(b + off[18]);
    h->d_st = (IterState *)(b + off[19]);
    h->d_cfg = (IterConfig *)(b + off[20]);
    h->loop_partials = (double *)(b + off[28]);
    h->loop_bar = (unsigned *)(b + off[29]);
    h->q_dev = (double *)(b + off[30]);
    h->dx_dev = (double *)(b + off[31]);
    if (h->prec == OCI_FP32) {
        h->ref_tab = (double *)(b + off[21]);
        h->ref_par = (double *)(b + off[22]);
        h->ref_muw = (double *)(b + off[23]);
        h->ref_h0P = b + off[24];
        h->ref_h0M = b + off[25];
        h->ref_r0 = b + off[26];
        h->ref_phi = b + off[27];
        if (h->staged && h->ks.cells_lin_tma) {
            h->cells_lin = h->ks.cells_lin_tma;
            h->cfg.stall_floor = 1e-5;
            if (const char *e = std::getenv("OCI_STALL_FLOOR")) h->cfg.stall_floor = std::atof(e);
            if (const char *e = std::getenv("OCI_STALL_ITERS")) h->cfg.stall_iters = std::atoi(e);
            if (cudaFuncSetAttribute(h->cells_lin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->cells_smem) !=
                cudaSuccess) {
                oci_destroy(h);
                return OCI_ECUDA;
            }
        }
    }
    if (h->use_async) {
        // third face buffer pair, sync block + per-block completion flags, per-block partials
        const size_t tw = (size_t)h->cells_grid * (size_t)(h->cells_block / 32);
        const size_t fa = (face + 256 + 255) & ~(size_t)255;
        h->as_zero_bytes = (sizeof(ocik::AsyncSync) + tw * 4 + 15) & ~(size_t)15;
        const size_t zb = (h->as_zero_bytes + 255) & ~(size_t)255;
        if (cudaMalloc(&h->async_mem, 2 * fa + zb + 4 * tw * 3 * sizeof(double)) != cudaSuccess) {
            oci_destroy(h);
            return OCI_ENOMEM;
        }
        char *a = (char *)h->async_mem;
        h->faceP[2] = a;
        h->faceM[2] = a + fa;
        h->as = (ocik::AsyncSync *)(a + 2 * fa);
        h->as_done = (unsigned *)(a + 2 * fa + sizeof(ocik::AsyncSync));
        h->as_part = (double *)(a + 2 * fa + zb);
        if (cudaMemsetAsync(h->async_mem, 0, 2 * fa + zb, h->stream) != cudaSuccess) {
            oci_destroy(h);
            return OCI_ECUDA;
        }
    }
    if (cudaMallocHost(&h->h_st, sizeof(IterState)) != cudaSuccess) { oci_destroy(h); return OCI_ENOMEM; }
    if (cudaMemsetAsync(h->d_base, 0, total, h->stream) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
        oci_destroy(h);
        return OCI_ECUDA;
    }
    rc = build_tables(h);
    // cell widths for the source scaling (after the allocation was cleared)
    if (!rc && cudaMemcpyAsync(h->dx_dev, h->dx.data(), sizeof(double) * J, cudaMemcpyHostToDevice, h->stream) !=
                   cudaSuccess)
        rc = cuda_fail(h, cudaGetLastError(), "cell widths");
    if (!rc) rc = upload_source(h, p->q);
    if (!rc) rc = upload_boundaries(h, p->psi_bc_left, p->psi_bc_right);
    if (!rc) rc = load_state(h, p->psi0);
    if (!rc && cudaMemcpy(h->d_cfg, &h->cfg, sizeof(IterConfig), cudaMemcpyHostToDevice) != cudaSuccess) rc = OCI_ECUDA;
    h->cfg_dev = h->cfg;
    if (!rc && p->precision == OCI_FP32_BF16HALO) {
        rc = halo_setup(h);
        if (!rc) h->halo = OCI_HALO_BF16;
    }
    if (rc) { oci_destroy(h); return rc; }
    *out = h;
    return OCI_OK;
}

void oci_destroy(oci_handle *h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->exec_oci) cudaGraphExecDestroy(h->exec_oci);
    if (h->exec_si) cudaGraphExecDestroy(h->exec_si);
    if (h->graph_oci) cudaGraphDestroy(h->graph_oci);
    if (h->graph_si) cudaGraphDestroy(h->graph_si);
    if (h->exec_lin) cudaGraphExecDestroy(h->exec_lin);
    if (h->graph_lin) cudaGraphDestroy(h->graph_lin);
    if (h->exec_cont) cudaGraphExecDestroy(h->exec_cont);
    if (h->graph_cont) cudaGraphDestroy(h->graph_cont);
    if (h->exec_oci_h) cudaGraphExecDestroy(h->exec_oci_h);
    if (h->exec_oci_bar) cudaGraphExecDestroy(h->exec_oci_bar);
    if (h->graph_oci_bar) cudaGraphDestroy(h->graph_oci_bar);
    if (h->async_mem) cudaFree(h->async_mem);
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
    }
    for (cudaEvent_t e : {h->ev_done, h->ev_q_ready, h->ev_q_free, h->ev_snap[0], h->ev_snap[1], h->ev_d2h[0], h->ev_d2h[1]})
        if (e) cudaEventDestroy(e);
    for (double *ps : h->phi_snap)
        if (ps) cudaFree(ps);
    if (h->graph_oci_h) cudaGraphDestroy(h->graph_oci_h);
    if (h->hface_mem) cudaFree(h->hface_mem);
    if (h->nn_mem) cudaFree(h->nn_mem);
    dense_free(h);
    if (h->scan_mem) cudaFree(h->scan_mem);
    if (h->exec_be) cudaGraphExecDestroy(h->exec_be);
    if (h->graph_be) cudaGraphDestroy(h->graph_be);
    if (h->be_mem) cudaFree(h->be_mem);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->h_st) cudaFreeHost(h->h_st);
    if (h->rs_st) cudaFreeHost(h->rs_st);
    if (h->rs_mem) cudaFree(h->rs_mem);
    if (h->rs_up) cudaStreamDestroy(h->rs_up);
    for (int k = 0; k < 2; ++k)
        for (cudaEvent_t e : {h->rs_ev0[k], h->rs_ev1[k], h->rs_done[k], h->rs_ready[k], h->rs_free[k]})
            if (e) cudaEventDestroy(e);
    if (h->d_base) cudaFree(h->d_base);
    delete h;
}

int oci_set_source(oci_handle *h, const double *q)
{
    if (!h || !q) return OCI_EINVAL;
    CK(h, cudaSetDevice(h->device));
    if (!h->step_pending) return upload_source(h, q);
    // a step is running: stage the copy on the copy stream (once the last
    // scaling kernel has read q_dev); the next step scales it
    CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_q_free, 0));
    CK(h, cudaMemcpyAsync(h->q_dev, q, (size_t)h->J * 32, cudaMemcpyHostToDevice, h->copy_stream));
    CK(h, cudaEventRecord(h->ev_q_ready, h->copy_stream));
    h->q_pending = true;
    h->q_host_valid = false;
    return OCI_OK;
}

int oci_set_iteration(oci_handle *h, double tol, int32_t max_iter, int32_t commit_unconverged)
{
    if (!h || !(tol >= 0.0) || max_iter < 1) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    h->cfg.tol = tol;
    h->cfg.max_iter = max_iter;
    h->cfg.commit_unconverged = commit_unconverged ? 1 : 0;
    return set_device_cfg(h, h->cfg);
}

int oci_set_stream(oci_handle *h, void *cuda_stream)
{
    if (!h) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaStreamSynchronize(h->stream));
    h->stream = (cudaStream_t)cuda_stream;
    return OCI_OK;
}

int oci_set_wait_limits(oci_handle *h, uint32_t poll_limit, int32_t barrier_shortfall)
{
    if (!h || barrier_shortfall < 0) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    h->cfg.bar_poll_limit = poll_limit;
    h->cfg.bar_shortfall = barrier_shortfall;
    return OCI_OK;
}

int oci_set_halo(oci_handle *h, int32_t halo)
{
    if (!h || (halo != OCI_HALO_FP32 && halo != OCI_HALO_BF16)) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    if (halo == OCI_HALO_BF16 && !h->exec_oci_h) {
        const int rc = halo_setup(h);
        if (rc) return rc;
    }
    h->halo = halo;
    return OCI_OK;
}

int oci_set_guess(oci_handle *h, int32_t guess)
{
    if (!h || (guess != OCI_GUESS_PREVIOUS && guess != OCI_GUESS_EXTRAPOLATE)) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    h->cfg.extrap = guess == OCI_GUESS_EXTRAPOLATE ? 1 : 0;
    return set_device_cfg(h, h->cfg);
}

int oci_set_time_scheme(oci_handle *h, int32_t scheme)
{
    if (!h || (scheme != OCI_TIME_MB && scheme != OCI_TIME_BE)) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    if (scheme == OCI_TIME_BE && !h->be_mem) {
        const int rc = be_setup(h);
        if (rc) {
            if (h->be_mem) cudaFree(h->be_mem);
            h->be_mem = nullptr;
            return rc;
        }
    }
    if (scheme != h->scheme) h->guess_valid = false;  // faces rebuilt from the committed state
    h->scheme = scheme;
    return OCI_OK;
}

int oci_set_solver(oci_handle *h, int32_t solver)
{
    if (!h || (solver != OCI_SOLVER_WOODBURY && solver != OCI_SOLVER_DENSE)) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    if (solver == OCI_SOLVER_DENSE && !h->dense.mem) {
        const int rc = dense_setup(h);
        if (rc) {
            dense_free(h);
            return rc;
        }
    }
    h->solver = solver;
    return OCI_OK;
}

int oci_set_sweep(oci_handle *h, int32_t sweep)
{
    if (!h || (sweep != OCI_SWEEP_MARCH && sweep != OCI_SWEEP_SCAN)) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    if (sweep == h->sweep) return OCI_OK;
    if (sweep == OCI_SWEEP_SCAN && !h->scan_mem) {
        const int nseg = (h->J + ocik::SCAN_SEG - 1) / ocik::SCAN_SEG;
        if (nseg > 65535) return OCI_EINVAL;
        const size_t nch = 2 * (size_t)h->P, rs = rsize(h);
        const size_t a = ((nch * nseg * 6 * rs) + 255) & ~(size_t)255;
        if (cudaMalloc(&h->scan_mem, a + nch * nseg * 2 * rs) != cudaSuccess) {
            h->scan_mem = nullptr;
            return OCI_ENOMEM;
        }
        h->scan_nseg = nseg;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    // the SI step graph is rebuilt with the other sweep on the next step
    if (h->exec_si) cudaGraphExecDestroy(h->exec_si);
    if (h->graph_si) cudaGraphDestroy(h->graph_si);
    h->exec_si = nullptr;
    h->graph_si = nullptr;
    h->sweep = sweep;
    return OCI_OK;
}

int oci_step(oci_handle *h, oci_stats *st) { return run_step(h, false, st); }

int si_step(oci_handle *h, oci_stats *st) { return run_step(h, true, st); }

int oci_step_async(oci_handle *h)
{
    if (!h) return OCI_EINVAL;
    if (h->step_pending || h->nn_mode != OCI_NN_OFF || h->solver != OCI_SOLVER_WOODBURY || h->scheme != OCI_TIME_MB)
        return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    int rc = pipe_setup(h);
    if (!rc) rc = ensure_graphs(h);
    if (!rc) rc = apply_pending_source(h);
    if (rc) return rc;
    int launches = 0;
    if (!h->guess_valid) {
        if ((rc = launch_guess(h))) return rc;
        ++launches;
    }
    if ((rc = set_device_cfg(h, h->cfg))) return rc;
    const bool halo_graph = h->halo == OCI_HALO_BF16 && h->exec_oci_h && h->cfg.max_iter >= 4;
    CK(h, cudaEventRecord(h->ev0, h->stream));
    CK(h, cudaGraphLaunch(halo_graph ? h->exec_oci_h : h->exec_oci, h->stream));
    CK(h, cudaEventRecord(h->ev1, h->stream));
    CK(h, cudaMemcpyAsync(h->h_st, h->d_st, sizeof(IterState), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaEventRecord(h->ev_done, h->stream));
    h->step_pending = true;
    h->pend_halo = halo_graph;
    h->pend_async = !halo_graph && h->use_async;
    h->pend_launches = launches;
    return OCI_OK;
}

int oci_step_wait(oci_handle *h, oci_stats *st)
{
    if (!h) return OCI_EINVAL;
    if (!h->step_pending) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    h->step_pending = false;
    CK(h, cudaEventSynchronize(h->ev_done));
    CK(h, cudaStreamSynchronize(h->copy_stream));  // the moments copied out before this step
    IterState s = *h->h_st;
    const int unroll = (h->staged && h->pdl_graph) ? kUnroll : 1;
    int launches = h->pend_launches;
    if (h->pend_halo) launches += 6;
    else if (h->pend_async) launches += 2;
    else if (h->use_loop) launches += 2;  // begin, the loop (which commits)
    else launches += 2 + unroll * ((s.iter + unroll - 1) / unroll);
    int refined = 0;
    if (s.status == ocik::ST_STALL && h->cells_lin && h->ks.refine) {
        const int main_iters = s.iter;
        int rc = refine_step(h, &s);
        if (rc) return rc;
        refined = 1;
        launches += 2 + (s.iter - main_iters);
        CK(h, cudaEventRecord(h->ev1, h->stream));
        if ((rc = read_state(h, &s))) return rc;
    }
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->guess_valid = s.committed != 0;
    const int status = map_status(s.status);
    if (st) {
        st->iters = s.iter;
        st->status = status;
        st->residual = s.resid;
        st->seconds = ms * 1e-3;
        st->committed = s.committed;
        st->nn_accepts = 0;
        st->nn_rejects = 0;
        st->refined = refined;
        st->launches = launches;
    }
    return status;
}

int oci_fluxes_async(oci_handle *h, double *phi)
{
    if (!h || !phi) return OCI_EINVAL;
    CK(h, cudaSetDevice(h->device));
    int rc = pipe_setup(h);
    if (rc) return rc;
    const int k = h->snap_k;
    // snapshot on the handle's stream (after the last enqueued step), host copy on
    // the copy stream; the snapshot is reused once its previous host copy is done
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_d2h[k], 0));
    CK(h, cudaMemcpyAsync(h->phi_snap[k], h->phi_out, (size_t)h->J * 32, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaEventRecord(h->ev_snap[k], h->stream));
    CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_snap[k], 0));
    CK(h, cudaMemcpyAsync(phi, h->phi_snap[k], (size_t)h->J * 32, cudaMemcpyDeviceToHost, h->copy_stream));
    CK(h, cudaEventRecord(h->ev_d2h[k], h->copy_stream));
    h->snap_k = k ^ 1;
    return OCI_OK;
}

int oci_sync(oci_handle *h)
{
    if (!h) return OCI_EINVAL;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->copy_stream) CK(h, cudaStreamSynchronize(h->copy_stream));
    return OCI_OK;
}

int oci_run_steps(oci_handle *h, int32_t n, const double *q, double *phi, oci_stats *stats, int32_t *done)
{
    if (!h || n < 0) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    if (done) *done = 0;
    const size_t Jq = (size_t)h->J * 4;
    auto skip_from = [&](int k0) {
        for (int k = k0; stats && k < n; ++k) {
            stats[k] = oci_stats{};
            stats[k].status = OCI_ESKIPPED;
        }
    };
    if (!queue_capable(h)) {  // one step at a time, as oci_set_source / oci_step / oci_fluxes
        for (int k = 0; k < n; ++k) {
            int rc = q ? upload_source(h, q + (size_t)k * Jq) : OCI_OK;
            if (rc) return rc;
            oci_stats st{};
            const int status = run_step(h, false, &st);
            if (stats) stats[k] = st;
            if (!st.committed) {
                skip_from(k + 1);
                return status == OCI_OK ? OCI_ENOTCONV : status;
            }
            if (phi && (rc = oci_fluxes(h, phi + (size_t)k * Jq))) return rc;
            if (done) *done = k + 1;
        }
        return OCI_OK;
    }
    int rc = pipe_setup(h);
    if (!rc) rc = ensure_graphs(h);
    if (!rc) rc = rs_setup(h);
    if (!rc) rc = apply_pending_source(h);
    if (!rc) rc = set_device_cfg(h, h->cfg);
    if (rc) return rc;
    if (n == 0) return OCI_OK;
    StepRange range("oci_run_steps");
    const int grid = std::min((h->J + 255) / 256, 152 * 8);
    int launches[2] = {0, 0};
    // the cell sources from the source moments staged in a slot (a slot's staging
    // buffer keeps its step's moments until the step two after it is enqueued)
    auto rescale = [&](int slot) -> int {
        k_scale_source<float><<<grid, 256, 0, h->stream>>>(h->rs_stage[slot], h->dx_dev, h->J, (r4<float> *)h->cellq);
        CK(h, cudaGetLastError());
        CK(h, cudaEventRecord(h->rs_free[slot], h->stream));  // the next upload into the slot waits for this read
        return OCI_OK;
    };
    // step k in slot k & 1: its source staged and scaled, [the initial iterate],
    // the step, its moments copied out; `behind`: queued behind step k - 1
    auto enqueue = [&](int k, bool behind) -> int {
        const int slot = k & 1;
        int r = OCI_OK;
        launches[slot] = 2;  // prologue, the loop (which commits)
        if (q) {
            CK(h, cudaStreamWaitEvent(h->rs_up, h->rs_free[slot], 0));
            CK(h, cudaMemcpyAsync(h->rs_stage[slot], q + (size_t)k * Jq, Jq * 8, cudaMemcpyHostToDevice, h->rs_up));
            CK(h, cudaEventRecord(h->rs_ready[slot], h->rs_up));
            CK(h, cudaStreamWaitEvent(h->stream, h->rs_ready[slot], 0));
            if ((r = rescale(slot))) return r;
            ++launches[slot];
        }
        if (!behind && !h->guess_valid) {
            if ((r = launch_guess(h))) return r;
            ++launches[slot];
        }
        r = rs_launch(h, slot, behind);
        if (!r && phi) r = rs_snapshot(h, slot, phi + (size_t)k * Jq);
        return r;
    };
    int status = OCI_OK, src_slot = (n - 1) & 1;  // slot whose staged source the cell sources hold at the end
    if ((rc = enqueue(0, false))) return rc;
    int queued_to = 1;  // steps enqueued
    for (int k = 0; k < n; ++k) {
        const int slot = k & 1, nslot = slot ^ 1;
        if (queued_to < n && queued_to == k + 1) {
            if ((rc = enqueue(queued_to, true))) return rc;
            ++queued_to;
        }
        const bool queued = queued_to == k + 2;  // step k + 1 is on the stream behind this one
        CK(h, cudaEventSynchronize(h->rs_done[slot]));
        IterState s = h->rs_st[slot];
        int refined = 0, lc = launches[slot];
        if (s.status == ocik::ST_STALL && h->cells_lin && h->ks.refine) {
            if (queued) {
                CK(h, cudaEventSynchronize(h->rs_done[nslot]));  // held behind this step: it did nothing
                if (q && (rc = rescale(slot))) return rc;         // this step's cell sources for its refinement
            }
            const int main_iters = s.iter;
            if ((rc = refine_step(h, &s))) return rc;
            refined = 1;
            lc += 2 + (s.iter - main_iters);
            CK(h, cudaEventRecord(h->rs_ev1[slot], h->stream));
            if ((rc = read_state(h, &s))) return rc;
            if (phi && s.committed && (rc = rs_snapshot(h, slot, phi + (size_t)k * Jq))) return rc;
            if (queued) {
                if (q && (rc = rescale(nslot))) return rc;
                if (s.committed) {  // the held step again, now behind a committed one
                    if ((rc = rs_launch(h, nslot, false))) return rc;
                    launches[nslot] += 2;
                    if (phi && (rc = rs_snapshot(h, nslot, phi + (size_t)(k + 1) * Jq))) return rc;
                }
            }
        }
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->rs_ev0[slot], h->rs_ev1[slot]));
        h->guess_valid = s.committed != 0;
        const int code = map_status(s.status);
        if (stats) {
            oci_stats &o = stats[k];
            o = oci_stats{};
            o.iters = s.iter;
            o.status = code;
            o.residual = s.resid;
            o.seconds = ms * 1e-3;
            o.committed = s.committed;
            o.refined = refined;
            o.launches = lc;
        }
        if (!s.committed) {
            status = code == OCI_OK ? OCI_ENOTCONV : code;
            if (queued) {
                CK(h, cudaEventSynchronize(h->rs_done[nslot]));  // held: it did nothing
                if (q && (rc = rescale(slot))) return rc;         // the handle keeps this step's sources
            }
            src_slot = slot;
            skip_from(k + 1);
            break;
        }
        if (done) *done = k + 1;
    }
    if (q) {  // the source moments of the cell sources now in place (as oci_set_source leaves them)
        CK(h, cudaMemcpyAsync(h->q_dev, h->rs_stage[src_slot], Jq * 8, cudaMemcpyDeviceToDevice, h->stream));
        h->q_host_valid = false;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaStreamSynchronize(h->copy_stream));
    CK(h, cudaStreamSynchronize(h->rs_up));
    return status;
}

int oci_fluxes(const oci_handle *hc, double *phi)
{
    oci_handle *h = const_cast<oci_handle *>(hc);
    if (!h || !phi) return OCI_EINVAL;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaMemcpyAsync(phi, h->phi_out, (size_t)h->J * 32, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return OCI_OK;
}

int oci_fluxes_device(const oci_handle *hc, void *dptr)
{
    oci_handle *h = const_cast<oci_handle *>(hc);
    if (!h || !dptr) return OCI_EINVAL;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaMemcpyAsync(dptr, h->phi_out, (size_t)h->J * 32, cudaMemcpyDeviceToDevice, h->stream));
    return OCI_OK;
}

int oci_get_state(const oci_handle *hc, double *psi)
{
    oci_handle *h = const_cast<oci_handle *>(hc);
    if (!h || !psi) return OCI_EINVAL;
    CK(h, cudaSetDevice(h->device));
    const int J = h->J, N = h->N, P = h->P;
    const size_t n = (size_t)J * P * 4;
    std::vector<double> pe(n);
    if (h->prec == OCI_FP64) {
        CK(h, cudaMemcpyAsync(pe.data(), h->psi_edge, n * 8, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    } else {
        std::vector<float> f(n);
        CK(h, cudaMemcpyAsync(f.data(), h->psi_edge, n * 4, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        for (size_t i = 0; i < n; ++i) pe[i] = f[i];
    }
    for (int j = 0; j < J; ++j)
        for (int p = 0; p < P; ++p) {
            const double *o = &pe[((size_t)j * P + p) * 4];
            const int mp = P + p, mm = P - 1 - p;
            psi[((size_t)j * N + mp) * 2] = o[0];
            psi[((size_t)j * N + mp) * 2 + 1] = o[1];
            psi[((size_t)j * N + mm) * 2] = o[2];
            psi[((size_t)j * N + mm) * 2 + 1] = o[3];
        }
    return OCI_OK;
}

int oci_set_state(oci_handle *h, const double *psi)
{
    if (!h || !psi) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    return load_state(h, psi);
}

int oci_dd_begin(oci_handle *h)
{
    if (!h) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    if (h->solver != OCI_SOLVER_WOODBURY || h->scheme != OCI_TIME_MB) return OCI_EINVAL;
    CK(h, cudaSetDevice(h->device));
    int rc = apply_pending_source(h);
    if (rc) return rc;
    if (!h->guess_valid && (rc = launch_guess(h))) return rc;
    // the step ends only by oci_dd_decide: no tolerance, count or stall exit on the device
    IterConfig c = h->cfg;
    c.tol = 0.0;
    c.max_iter = 0x3fffffff;
    c.stall_floor = 0.0;
    c.pause_at = -1;
    if ((rc = set_device_cfg(h, c))) return rc;
    CK(h, cudaEventRecord(h->ev0, h->stream));
    IterState *st = h->d_st;
    void *a_st[] = {&st};
    CK(h, cudaLaunchKernel((const void *)&ocik::k_step_begin, dim3(1), dim3(1), a_st, 0, h->stream));
    h->dd_active = true;
    h->dd_iter = 0;
    return OCI_OK;
}

int oci_dd_export(oci_handle *h, void *out_left, void *out_right)
{
    if (!h) return OCI_EINVAL;
    if (!h->dd_active) return OCI_ESTATE;
    return dd_faces(h, out_left, out_right, 0);
}

int oci_dd_import(oci_handle *h, const void *in_left, const void *in_right)
{
    if (!h) return OCI_EINVAL;
    if (!h->dd_active) return OCI_ESTATE;
    return dd_faces(h, const_cast<void *>(in_left), const_cast<void *>(in_right), 1);
}

int oci_dd_iterate(oci_handle *h, double *sums)
{
    if (!h || !sums) return OCI_EINVAL;
    if (!h->dd_active) return OCI_ESTATE;
    int rc = dd_iteration(h);
    IterState s{};
    if (!rc) rc = read_state(h, &s);
    if (rc) return rc;
    ++h->dd_iter;
    sums[0] = s.d2;
    sums[1] = s.p2;
    return OCI_OK;
}

int oci_dd_decide(oci_handle *h, const double *sums, int32_t *done, oci_stats *stats)
{
    if (!h || !sums || !done) return OCI_EINVAL;
    if (!h->dd_active || h->dd_iter < 1) return OCI_ESTATE;
    const double a = sums[0], b = sums[1];
    double resid;
    if (b > 0.0) resid = std::sqrt(a / b);
    else resid = a == 0.0 ? 0.0 : INFINITY;
    int ns = ocik::ST_RUNNING;
    if (!(resid == resid) || !(a == a) || !(b == b) || std::isinf(b)) ns = ocik::ST_NAN;
    else if (resid < h->cfg.tol) ns = ocik::ST_CONVERGED;
    else if (h->dd_iter >= h->cfg.max_iter) ns = ocik::ST_MAXITER;
    *done = ns != ocik::ST_RUNNING;
    if (!*done) return OCI_OK;
    void *a_dec[] = {&h->d_st, &ns, &resid, const_cast<double *>(&a), const_cast<double *>(&b)};
    CK(h, cudaLaunchKernel((const void *)&k_dd_decide, dim3(1), dim3(1), a_dec, 0, h->stream));
    KParams<double> pd = make_params<double>(h, 0, 0);
    KParams<float> pf = make_params<float>(h, 0, 0);
    void *args[] = {h->prec == OCI_FP64 ? (void *)&pd : (void *)&pf};
    CK(h, cudaLaunchKernel(h->ks.commit_oci, dim3(h->grid_pc), dim3(kBlock), args, 0, h->stream));
    CK(h, cudaEventRecord(h->ev1, h->stream));
    IterState s{};
    int rc = read_state(h, &s);
    if (rc) return rc;
    h->dd_active = false;
    h->guess_valid = s.committed != 0;
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    const int status = map_status(s.status);
    if (stats) {
        *stats = oci_stats{};
        stats->iters = s.iter;
        stats->status = status;
        stats->residual = resid;
        stats->seconds = ms * 1e-3;
        stats->committed = s.committed;
        stats->launches = 3 + 3 * h->dd_iter;  // begin, decision, commit; per iteration import, export, cells
    }
    return status;
}

int oci_profile_iterations(oci_handle *h, int32_t n_iter, double *seconds_per_launch)
{
    if (!h || n_iter < 1 || !seconds_per_launch) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    int rc = launch_guess(h);
    if (rc) return rc;
    // no exit on tolerance or iteration count while timing
    IterConfig timing{};
    timing.max_iter = 0x3fffffff;
    timing.tol = 0.0;
    timing.commit_unconverged = 0;
    int rc0 = set_device_cfg(h, timing);
    if (rc0) return rc0;
    IterState *st = h->d_st;
    void *a_st[] = {&st};
    CK(h, cudaLaunchKernel((const void *)&ocik::k_step_begin, dim3(1), dim3(1), a_st, 0, h->stream));
    if (h->scheme == OCI_TIME_BE) {
        // the backward-Euler iteration kernel as plain launches
        const int grid = std::max(1, std::min((h->J + 7) / 8, h->grid_cells));
        KParams<double> bd = make_params<double>(h, 0, 0);
        KParams<float> bf = make_params<float>(h, 0, 0);
        ocik::BeArgs<double> ad{(const r2<double> *)h->be_tab, h->be_K, h->be_Kf};
        ocik::BeArgs<float> af{(const r2<float> *)h->be_tab, h->be_K, h->be_Kf};
        void *ba[] = {h->prec == OCI_FP64 ? (void *)&bd : (void *)&bf, h->prec == OCI_FP64 ? (void *)&ad : (void *)&af};
        for (int i = -2; i < n_iter; ++i) {
            if (i == 0) CK(h, cudaEventRecord(h->ev0, h->stream));
            CK(h, cudaLaunchKernel(h->ks.be_cells, dim3(grid), dim3(kBlock), ba, 0, h->stream));
        }
        CK(h, cudaEventRecord(h->ev1, h->stream));
        CK(h, cudaEventSynchronize(h->ev1));
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        *seconds_per_launch = ms * 1e-3 / n_iter;
        if ((rc = set_device_cfg(h, h->cfg))) return rc;
        h->guess_valid = false;
        return OCI_OK;
    }
    if (h->use_loop && h->solver == OCI_SOLVER_WOODBURY) {
        // the persistent loop: one cooperative launch runs a fixed number of iterations
        auto prepare = [&]() -> int {
            CK(h, cudaLaunchKernel((const void *)&ocik::k_step_begin, dim3(1), dim3(1), a_st, 0, h->stream));
            CK(h, cudaMemsetAsync(h->loop_bar, 0, sizeof(unsigned), h->stream));
            if (h->use_async) CK(h, cudaMemsetAsync(h->as, 0, h->as_zero_bytes, h->stream));
            return OCI_OK;
        };
        auto launch = [&](int n) -> int {  // the loop a step runs (barrier-free where available)
            h->loop_fixed = n;
            KParams<float> pl = make_params<float>(h, 0, 0);
            h->loop_fixed = 0;
            void *la[] = {&pl};
            CK(h, cudaLaunchCooperativeKernel(h->use_async ? h->cells_async : h->cells_loop, dim3(h->cells_grid),
                                              dim3(h->cells_block), la, h->cells_smem, h->stream));
            return OCI_OK;
        };
        if (h->halo == OCI_HALO_BF16) {
            // the BF16 phase's loop, after its entry iteration (which it needs for its faces)
            auto entry = [&]() -> int {
                KParams<float> pe = make_params<float>(h, 0, 0);
                void *ea[] = {&pe};
                CK(h, cudaLaunchKernel(h->hk.entry, dim3(h->cells_grid), dim3(h->cells_block), ea, h->cells_smem,
                                       h->stream));
                CK(h, cudaMemsetAsync(h->loop_bar, 0, sizeof(unsigned), h->stream));
                return OCI_OK;
            };
            auto hlaunch = [&](int n) -> int {
                h->loop_fixed = n + 1;  // the entry iteration counts
                KParams<float> pl = make_params<float>(h, 0, 0);
                h->loop_fixed = 0;
                void *la[] = {&pl};
                CK(h, cudaLaunchCooperativeKernel(h->hk.loop, dim3(h->cells_grid), dim3(h->cells_block), la,
                                                  h->cells_smem, h->stream));
                return OCI_OK;
            };
            if ((rc = prepare()) || (rc = entry()) || (rc = hlaunch(2)) || (rc = prepare()) || (rc = entry())) return rc;
            CK(h, cudaEventRecord(h->ev0, h->stream));
            if ((rc = hlaunch(n_iter))) return rc;
            CK(h, cudaEventRecord(h->ev1, h->stream));
            CK(h, cudaEventSynchronize(h->ev1));
            float ms = 0.f;
            CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
            *seconds_per_launch = ms * 1e-3 / n_iter;
            if ((rc = set_device_cfg(h, h->cfg))) return rc;
            h->guess_valid = false;
            return OCI_OK;
        }
        if ((rc = prepare()) || (rc = launch(2)) || (rc = prepare())) return rc;  // warm-up
        CK(h, cudaEventRecord(h->ev0, h->stream));
        if ((rc = launch(n_iter))) return rc;
        CK(h, cudaEventRecord(h->ev1, h->stream));
        CK(h, cudaEventSynchronize(h->ev1));
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        *seconds_per_launch = ms * 1e-3 / n_iter;
        if ((rc = set_device_cfg(h, h->cfg))) return rc;
        h->guess_valid = false;
        return OCI_OK;
    }
    KParams<double> pd = make_params<double>(h, 0, 0);
    KParams<float> pf = make_params<float>(h, 0, 0);
    void *args[] = {h->prec == OCI_FP64 ? (void *)&pd : (void *)&pf};
    for (int i = -2; i < n_iter; ++i) {  // two untimed warm-up launches (library setup, caches)
        if (i == 0) CK(h, cudaEventRecord(h->ev0, h->stream));
        if (h->solver == OCI_SOLVER_DENSE) {
            if ((rc = dense_iterate(h))) return rc;
        } else if (h->staged) {
            cudaLaunchConfig_t lc{};
            lc.gridDim = dim3(h->cells_grid);
            lc.blockDim = dim3(h->cells_block);
            lc.dynamicSmemBytes = h->cells_smem;
            lc.stream = h->stream;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            lc.attrs = at;
            lc.numAttrs = 1;
            CK(h, cudaLaunchKernelExC(&lc, h->cells_oci, args));
        } else {
            CK(h, cudaLaunchKernel(h->cells_oci, dim3(h->cells_grid), dim3(h->cells_block), args, h->cells_smem,
                                   h->stream));
        }
    }
    CK(h, cudaEventRecord(h->ev1, h->stream));
    CK(h, cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    *seconds_per_launch = ms * 1e-3 / n_iter;
    if ((rc = set_device_cfg(h, h->cfg))) return rc;
    h->guess_valid = false;  // the face buffers now hold timing iterates
    return OCI_OK;
}

int oci_nn_attach(oci_handle *h, const float *params, int32_t mode, int32_t k_corr)
{
    if (!h || mode < OCI_NN_OFF || mode > OCI_NN_GUESS_ADAPTIVE) return OCI_EINVAL;
    if (mode != OCI_NN_OFF && (!params || k_corr < 1)) return OCI_EINVAL;
    if (h->step_pending || h->dd_active) return OCI_ESTATE;
    CK(h, cudaSetDevice(h->device));
    if (mode == OCI_NN_OFF) {
        h->nn_mode = OCI_NN_OFF;
        return OCI_OK;
    }
    const int J = h->J;
    const size_t npar = (size_t)oci_nn_param_count();
    if (!h->nn_mem) {
        const size_t ws = oci_nn_workspace_bytes(1, J);
        size_t sizes[] = {npar * 4, (size_t)J * 13 * 4, (size_t)J * 16, 256, (size_t)J * 16, (size_t)J * 4,
                          (size_t)J * 32, (size_t)J * 32, (size_t)J * 32, (size_t)J * 32, ws, 2 * face_bytes(h)};
        size_t off[12], total = 0;
        for (int i = 0; i < 12; ++i) {
            off[i] = total;
            total += (sizes[i] + 255) & ~(size_t)255;
        }
        if (cudaMalloc(&h->nn_mem, total) != cudaSuccess) return OCI_ENOMEM;
        char *b = (char *)h->nn_mem;
        h->nn_params = (float *)(b + off[0]);
        h->nn_in = (float *)(b + off[1]);
        h->nn_out = (float *)(b + off[2]);
        h->nn_scale = (float *)(b + off[3]);
        h->nn_stat = (float *)(b + off[4]);
        h->nn_qfeat = (float *)(b + off[5]);
        h->nn_phat = (double *)(b + off[6]);
        h->nn_hist[0] = (double *)(b + off[7]);
        h->nn_hist[1] = (double *)(b + off[8]);
        h->nn_phi_bak = (double *)(b + off[9]);
        h->nn_ws = b + off[10];
        h->nn_ws_bytes = ws;
        h->nn_face_bak = b + off[11];
        std::vector<float> st, qf;
        if (int rq = sync_q_host(h)) return rq;
        nn_host_features(h, st, qf);
        CK(h, cudaMemcpy(h->nn_stat, st.data(), sizeof(float) * st.size(), cudaMemcpyHostToDevice));
        CK(h, cudaMemcpy(h->nn_qfeat, qf.data(), sizeof(float) * qf.size(), cudaMemcpyHostToDevice));
        // history starts at the current committed moments (both entries)
        CK(h, cudaStreamSynchronize(h->stream));
        CK(h, cudaMemcpy(h->nn_hist[0], h->phi_out, (size_t)J * 32, cudaMemcpyDeviceToDevice));
        CK(h, cudaMemcpy(h->nn_hist[1], h->phi_out, (size_t)J * 32, cudaMemcpyDeviceToDevice));
    }
    CK(h, cudaMemcpy(h->nn_params, params, npar * 4, cudaMemcpyHostToDevice));
    h->nn_mode = mode;
    h->nn_kcorr = k_corr;
    h->nn_trial = -2;  // two plain steps first: the start of a run is often a transient
    h->nn_trial_plain = h->nn_trial_nn = 0;
    h->nn_use = true;
    h->nn_since_trial = 0;
    return OCI_OK;
}

int oci_nn_static_features(const oci_handle *hc, void *stat, void *qfeat)
{
    oci_handle *h = const_cast<oci_handle *>(hc);
    if (!h || !stat || !qfeat) return OCI_EINVAL;
    CK(h, cudaSetDevice(h->device));
    if (int rq = sync_q_host(h)) return rq;
    std::vector<float> st, qf;
    nn_host_features(h, st, qf);
    CK(h, cudaMemcpy(stat, st.data(), sizeof(float) * st.size(), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(qfeat, qf.data(), sizeof(float) * qf.size(), cudaMemcpyHostToDevice));
    return OCI_OK;
}

int oci_query(const oci_handle *h, int32_t *n_cells, int32_t *n_ord, double *mu, double *w)
{
    if (!h) return OCI_EINVAL;
    if (n_cells) *n_cells = h->J;
    if (n_ord) *n_ord = h->N;
    if (mu) std::memcpy(mu, h->mu.data(), sizeof(double) * h->N);
    if (w) std::memcpy(w, h->w.data(), sizeof(double) * h->N);
    return OCI_OK;
}

const char *oci_strerror(int code)
{
    switch (code) {
    case OCI_OK: return "ok";
    case OCI_EINVAL: return "invalid argument";
    case OCI_ENOMEM: return "out of memory";
    case OCI_ECUDA: return "CUDA error";
    case OCI_ENOTCONV: return "not converged within max_iter";
    case OCI_ENAN: return "non-finite scalar flux";
    case OCI_ETIMEOUT: return "device iteration guard tripped";
    case OCI_ESTATE: return "call not valid in this state";
    case OCI_ESKIPPED: return "step not run: an earlier step of the call did not commit";
    default: return "unknown status";
    }
}

const char *oci_last_cuda_error(const oci_handle *h) { return h ? h->err.c_str() : ""; }

}  // extern "C"
