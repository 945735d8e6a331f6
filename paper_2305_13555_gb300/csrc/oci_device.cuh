// Device code for the one-cell-inversion (OCI) and source-iteration (SI)
// schemes of MB-SCB transient slab S_N transport (arXiv 2305.13555).
//
// Data layout in HBM (R = float in FP32 mode, double in FP64 mode; P = N/2
// ordinate pairs, pair p = (mu_p > 0, -mu_p), ascending mu_p):
//   faceP[b][f][p]   r2  outgoing flux of +mu_p through face f (f = 0..J), the
//                        (k, k+1/2) values of the upstream corner R of cell f-1;
//   faceM[b][f][p]   r2  outgoing flux of -mu_p through face f, corner L of cell f;
//                        b = ping-pong buffer; faceP[b][0] / faceM[b][J] hold
//                        the prescribed boundary data and are never written by
//                        a cell.
//   psi_edge[j][p]   r4  time-edge flux psi_{k-1/2}: (+L, +R, -L, -R)
//   cellq[j]         r4  (dx/4) (Q_kL, Q_kR, Q_hL, Q_hR)
//   mat[j]           int material id; tab[m][p] = complex entries of A_{+mu}^{-1};
//                        matpar[m] = (e = dx/(2 v dt), s = dx Sigma_s / 4);
//                        matK[m] = (I - s M)^{-1} in double (Woodbury capacitance)
//   phi[2][j][4]     scalar-flux moment iterates, ping-pong (double in FP64
//                        mode, double-float (h, l) pairs in FP32 mode)
//   g[p][j]          r4  SI affine offsets (pair-major for the march)
//   refl[p]          r2  SI: +mu flux leaving x = X in the previous iterate
//
// Per ordinate the 4x4 block of the SI section, A_m, acts on the corner pair
// (L, R) as multiplication by a complex number: with v = v_L + i v_R the
// streaming/collision block [[a, mu/2], [-mu/2, a]] is t = a - i mu/2, so
//   A_{+mu} = [[t, e], [-2e, t + 2e]]  (a 2x2 matrix over C),
//   A_{+mu}^{-1} = [[t + 2e, -e], [2e, t]] / (t (t + 2e) + 2 e^2),
//   A_{-mu} = conj(A_{+mu}).
// The cell system (A - S) Psi = c of the OCI section has S = s (1 w^T) (x) I_4,
// so with y_m = A_m^{-1} c_m, r = sum_m w_m y_m, M = sum_m w_m A_m^{-1}:
//   phi = (I - s M)^{-1} r,   psi_m = y_m + s A_m^{-1} phi   (Woodbury).
// For a symmetric quadrature M is real in the C sense (M = M_r (x) I_2), so the
// capacitance solve is two 2x2 real systems sharing one inverse K.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ocik {

constexpr unsigned FULL = 0xffffffffu;

template <typename R> struct __align__(2 * sizeof(R)) r2 { R x, y; };
template <typename R> struct __align__(16) r4 { R x, y, z, w; };
struct __align__(16) kmat { double k00, k01, k10, k11; };

enum : int { BC_VACUUM = 0, BC_REFLECT = 1, BC_INCIDENT = 2 };
enum : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_MAXITER = 2, ST_NAN = 3, ST_GUARD = 4, ST_TIMEOUT = 5, ST_STALL = 6,
             ST_SWITCH = 7, ST_HELD = 8 };  // ST_SWITCH: the BF16-halo phase of a step ended, FP32 iterations follow
// k_cells modes (M_LIN: correction equation of the FP32 refinement, staged kernel only)
enum : int { M_OCI = 0, M_SI = 1, M_LIN = 2 };
// k_percell modes
enum : int { C_COMMIT_OCI = 0, C_COMMIT_SI = 1, C_SI_PREP = 2, C_GUESS = 3, C_COMMIT_LIN = 4 };

// Iteration state of the current time step (device memory, one per handle).
struct IterState {
    int iter;          // iterations completed in this step
    int status;        // ST_*
    int base;          // face buffer read by iteration 1 of this step
    int base_next;     // face buffer holding the next step's initial iterate
    unsigned int arrive;  // blocks of the current launch that finished
    int launches;      // launches of the iteration kernel in this step (guard)
    int committed;     // last step advanced the state
    int stall;         // iterations since the relative change last fell by 10%
    double resid;      // last relative change of phi
    double d2, p2;     // sum (dphi)^2, sum phi^2 of the last iteration
    double best;       // smallest relative change since the last 10% improvement
    int rot3;          // this step's iterations rotated through three face buffers
    int cur_face;      // ... and the buffer holding the latest iterate
    int lin_first;     // FP32 refinement: number of the correction's first iteration
    int chain;         // set before a step queued behind another: hold it unless that one committed
};

// Barrier-free persistent loop (k_cells_tma ASYNC): per-iteration arrival
// counters and decisions, in a ring of four iterations.  Zeroed before each
// launch together with the per-block completion flags that follow it.
struct AsyncRec {
    double resid, d2, p2, best;
    int status, stall, pad0, pad1;
};
struct AsyncSync {
    unsigned cnt[4];      // blocks that finished iteration rep (slot rep & 3), cumulative
    unsigned tag[4];      // rep + 1 once the decision of iteration rep is in rec[rep & 3]
    unsigned exit_bar;    // blocks that reached the end of the launch
    unsigned pad[7];
    AsyncRec rec[4];
};

struct IterConfig {
    int max_iter;
    int commit_unconverged;
    double tol;
    int pause_at;      // iteration count at which the loop stops with the step still running (-1: never)
    int stall_iters;   // stop with ST_STALL after this many iterations without a 10% improvement ...
    double stall_floor;  // ... once the relative change is below this (0 disables)
    unsigned bar_poll_limit;  // grid-barrier polls before a timeout (0: kWaitLimit)
    int bar_shortfall;        // arrivals the grid barrier waits for beyond the grid (diagnostic; 0)
    double halo_switch;       // BF16-halo phase: leave it once the relative change is below this ...
    int halo_stall;           // ... or after this many iterations without a 10% improvement
    int extrap;               // next step's initial iterate: 0 the end-of-step flux, 1 its extrapolation in time
};


// ------------------------------------------------------------ load helpers
__device__ __forceinline__ r4<float> ldg4(const r4<float> *p)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ r4<double> ldg4(const r4<double> *p)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ r2<float> ldg2(const r2<float> *p)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ r2<double> ldg2(const r2<double> *p)
{
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return {v.x, v.y};
}
// Streaming (read-write across launches) data: plain coherent loads.
__device__ __forceinline__ r4<float> ld4(const r4<float> *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ r4<double> ld4(const r4<double> *p)
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ r2<float> ld2(const r2<float> *p)
{
    const float2 v = *reinterpret_cast<const float2 *>(p);
    return {v.x, v.y};
}
__device__ __forceinline__ r2<double> ld2(const r2<double> *p)
{
    const double2 v = *reinterpret_cast<const double2 *>(p);
    return {v.x, v.y};
}
template <typename R> __device__ __forceinline__ void st2(r2<R> *p, R x, R y) { *p = r2<R>{x, y}; }

// Loads through L2 only (data another SM may have written during the launch).
__device__ __forceinline__ r2<float> ldcg2(const r2<float> *p)
{
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ r2<double> ldcg2(const r2<double> *p)
{
    const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ r4<float> ldcg4(const r4<float> *p)
{
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ r4<double> ldcg4(const r4<double> *p)
{
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}

// BF16 storage of a face pair (the (k, k+1/2) values of one ordinate at one
// face) in one 32-bit word: x in the low half, y in the high half, rounded to
// nearest even.  Widening is exact (a bf16 is the upper half of a float).
__device__ __forceinline__ unsigned pack_bf16x2(float x, float y)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<const unsigned *>(&v);
}
__device__ __forceinline__ r2<float> unpack_bf16x2(unsigned u)
{
    return r2<float>{__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u)};
}
template <typename R> __device__ __forceinline__ void st4(r4<R> *p, R x, R y, R z, R w) { *p = r4<R>{x, y, z, w}; }

// Complex entries of A_{+mu}^{-1} for one (material, pair).
template <typename R> struct Coef { R pr, pi, rr, ri, ur, ui, vr, vi; };

template <typename R>
__device__ __forceinline__ Coef<R> load_coef(const r4<R> *tab, int m, int P, int p)
{
    const r4<R> *t = tab + ((size_t)m * P + p) * 2;
    const r4<R> a = ldg4(t), b = ldg4(t + 1);
    return {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}

// y = A^{-1} u for the complex 2-vector u = (uk, uh).
template <typename R>
__device__ __forceinline__ void ainv(const Coef<R> &a, R ukr, R uki, R uhr, R uhi, R &ykr, R &yki, R &yhr, R &yhi)
{
    ykr = a.pr * ukr - a.pi * uki + a.rr * uhr - a.ri * uhi;
    yki = a.pr * uki + a.pi * ukr + a.rr * uhi + a.ri * uhr;
    yhr = a.ur * ukr - a.ui * uki + a.vr * uhr - a.vi * uhi;
    yhi = a.ur * uki + a.ui * ukr + a.vr * uhi + a.vi * uhr;
}

// Error-free sum (Knuth's TwoSum) in round-to-nearest.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    e = 0.0;
}

// Double-float ("FF") numbers: value = h + l with |l| <= ulp(h)/2, ~48-bit
// significand, built from FP32 operations with explicit rounding (Dekker /
// Knuth error-free transformations).  The FP32 path uses them where a double
// is needed -- the Woodbury capacitance solve and the iterate difference of
// the residual -- because FP64 throughput on this part is 1/58 of FP32.
struct ff { float h, l; };

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)  // requires |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_norm(float a, float b)
{
    float s, e;
    two_sum(a, b, s, e);
    return {s, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return ff_fast_two_sum(s, e);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ float ff_diff(ff a, ff b)  // (a - b) rounded to float
{
    return __fadd_rn(__fsub_rn(a.h, b.h), __fsub_rn(a.l, b.l));
}

// Storage of the scalar-flux iterates: double in FP64 mode, FF pairs (h, l)
// in FP32 mode (8 bytes either way).
template <typename R> struct PhiStore;
template <> struct PhiStore<double> {
    using S = double;
    static __device__ __forceinline__ double real(S v) { return v; }
    static __device__ __forceinline__ double wide(S v) { return v; }
};
template <> struct PhiStore<float> {
    using S = float2;
    static __device__ __forceinline__ float real(S v) { return __fadd_rn(v.x, v.y); }
    static __device__ __forceinline__ double wide(S v) { return (double)v.x + (double)v.y; }
};
template <typename R> using phi_t = typename PhiStore<R>::S;

// The 4 moments of one cell as R (for the s phi terms).
template <typename R>
__device__ __forceinline__ void load_phi4(const phi_t<R> *ph, int cell, R &a, R &b, R &c, R &d)
{
    const phi_t<R> *q = ph + 4 * (size_t)cell;
    a = PhiStore<R>::real(__ldcg(q));
    b = PhiStore<R>::real(__ldcg(q + 1));
    c = PhiStore<R>::real(__ldcg(q + 2));
    d = PhiStore<R>::real(__ldcg(q + 3));
}

template <typename R>
__device__ __forceinline__ phi_t<R> phi_from_double(double x);
template <> __device__ __forceinline__ double phi_from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float2 phi_from_double<float>(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

template <typename R>
struct KParams {
    int J, P;
    int bc_left, bc_right;
    int use_cond;
    int pad0;
    cudaGraphConditionalHandle cond;
    const int *mat;
    const r4<R> *cellq;
    const r4<R> *tab;      // [n_mat][P][2]: (Pr, Pi, Rr, Ri), (Ur, Ui, Vr, Vi)
    const r2<R> *matpar;   // [n_mat]: (e, s)
    const kmat *matK;      // [n_mat]
    const r2<R> *muw;      // [P]: (mu, w)
    r2<R> *faceP[3];       // [2]: third buffer of the barrier-free loop (or null)
    r2<R> *faceM[3];
    r4<R> *psi_edge;
    r4<R> *g;
    r2<R> *refl;           // [P] SI: lagged mirror flux at a reflecting right face
    phi_t<R> *phi[2];      // iterates l / l+1 (ping-pong)
    phi_t<R> *phi0;        // initial iterate of the step
    double *phi_out;       // published moments of the last committed step
    const float4 *matKf;   // [n_mat][2] FF capacitance (k00h,k00l,k01h,k01l),(k10h,k10l,k11h,k11l)
    // FP32 refinement: saved halo h0, its high-precision residual r0 (per producing
    // cell: +mu k, +mu k+1/2, -mu k, -mu k+1/2) and scalar flux phi(h0) (FF)
    const r2<R> *h0P, *h0M;
    const r4<R> *r0;
    const float2 *phi_ref;
    double *partials;      // [gridDim.x][2]
    IterState *st;
    const IterConfig *cfg;
    // persistent OCI loop: per-block (d2, p2, fault) of the last two iterations,
    // the grid barrier's arrival counter (zeroed before each launch), and a fixed
    // iteration count for timing (0: run to the iteration controls)
    double *loop_partials;
    unsigned *loop_bar;
    int loop_fixed;
    // persistent OCI loop: end the step in the same launch (commit after the
    // final decision) instead of a separate k_percell launch
    int loop_commit;
    // BF16-halo phase of the FP32 OCI iteration: the face buffers as bf16 pairs
    // (pack_bf16x2), same layout and ping-pong parity as faceP / faceM
    unsigned *hfP[2];
    unsigned *hfM[2];
    // barrier-free persistent loop: sync block, per-block completion flags
    // (iterations of this launch finished), per-block partials [4][blocks][3]
    AsyncSync *as;
    unsigned *as_done;
    double *as_part;
};

// Arithmetic of the end of a step with every rounding spelled out (no compiler
// contraction), so that every kernel that commits a step -- the per-cell
// commit, and the persistent loops that end the step in the same launch --
// produces the same bits from the same inputs.
__device__ __forceinline__ float mul_x(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_x(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_x(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_x(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float fma_x(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_x(double a, double b, double c) { return __fma_rn(a, b, c); }

// End-of-step (k+1/2) corner fluxes of ordinate pair (+mu, -mu) of one cell:
// the right-hand side from the source qd, the previous end-of-step flux pe
// (times e), the scattering terms F (already times s) and the incident faces
// inP / inM, then the second rows of the complex 2x2 inverse a.  Outputs:
// +mu (L, R) = (phr, phi), -mu (L, R) = (mhr, -mhi).
template <typename R>
__device__ __forceinline__ void commit_corners(const Coef<R> &a, const r4<R> &qd, R e, const r4<R> &pe, R Fkl,
                                               R Fkr, R Fhl, R Fhr, R mu, const r2<R> &inP, const r2<R> &inM,
                                               R &phr, R &phi, R &mhr, R &mhi)
{
    const R ukr = fma_x(mu, inP.x, add_x(fma_x(e, pe.x, qd.x), Fkl));
    const R uki = add_x(fma_x(e, pe.y, qd.y), Fkr);
    const R uhr = fma_x(mu, inP.y, add_x(qd.z, Fhl));
    const R uhi = add_x(qd.w, Fhr);
    const R vkr = add_x(fma_x(e, pe.z, qd.x), Fkl);
    const R vki = fma_x(-mu, inM.x, -add_x(fma_x(e, pe.w, qd.y), Fkr));
    const R vhr = add_x(qd.z, Fhl);
    const R vhi = fma_x(-mu, inM.y, -add_x(qd.w, Fhr));
    phr = fma_x(-a.vi, uhi, fma_x(a.vr, uhr, fma_x(-a.ui, uki, mul_x(a.ur, ukr))));
    phi = fma_x(a.vi, uhr, fma_x(a.vr, uhi, fma_x(a.ui, ukr, mul_x(a.ur, uki))));
    mhr = fma_x(-a.vi, vhi, fma_x(a.vr, vhr, fma_x(-a.ui, vki, mul_x(a.ur, vkr))));
    mhi = fma_x(a.vi, vhr, fma_x(a.vr, vhi, fma_x(a.ui, vkr, mul_x(a.ur, vki))));
}

// The previous end-of-step moments (entries 2, 3 of a cell's published phi)
// for every lane of the cell's segment (mask, its first lane base, lane ls in
// it): each is read by the lane that later overwrites it (lane c % LPC stores
// moment c), so the read precedes that store in the lane's own order, and
// shuffled to the others.
__device__ __forceinline__ void prev_end_moments(const double *phi_cell, unsigned mask, int base, int ls,
                                                 double &old2, double &old3)
{
    const int lpc = __popc(mask);
    const double v2 = ls == 2 % lpc ? __ldcg(phi_cell + 2) : 0.0;
    const double v3 = ls == 3 % lpc ? __ldcg(phi_cell + 3) : 0.0;
    old2 = __shfl_sync(mask, v2, base + 2 % lpc);
    old3 = __shfl_sync(mask, v3, base + 3 % lpc);
}

// Reduce V values per lane (s with compensation e) over the LPC lanes of a
// segment.  Afterwards lane holds NV = max(V/LPC, 1) sums in s[0..NV-1] for
// value indices [base, base + NV) with base = NV * (lane % LPC) when V >= LPC,
// else lane % V (lanes above V in the segment hold copies).
template <int LPC, int V, bool COMP, typename R>
__device__ __forceinline__ void reduce_scatter(R (&s)[V], R (&e)[V], int lane)
{
    constexpr int LS = LPC < V ? LPC : V;
    // all-reduce over the segment bits above LS (only when V < LPC)
#pragma unroll
    for (int o = LPC / 2; o >= LS && o >= 1; o >>= 1) {
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const R rs = __shfl_xor_sync(FULL, s[i], o);
            if constexpr (COMP) {
                const R re = __shfl_xor_sync(FULL, e[i], o);
                R t;
                two_sum(s[i], rs, s[i], t);
                e[i] = e[i] + re + t;
            } else {
                s[i] = s[i] + rs;
            }
        }
    }
    // reduce-scatter over the low log2(LS) bits
#pragma unroll
    for (int lev = 0; (LS >> (lev + 1)) >= 1; ++lev) {
        const int o = LS >> (lev + 1);
        const int half = V >> (lev + 1);
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const R snd = up ? s[i] : s[i + half];
            const R kp = up ? s[i + half] : s[i];
            const R rs = __shfl_xor_sync(FULL, snd, o);
            if constexpr (COMP) {
                const R esnd = up ? e[i] : e[i + half];
                const R ekp = up ? e[i + half] : e[i];
                const R re = __shfl_xor_sync(FULL, esnd, o);
                R t;
                two_sum(kp, rs, s[i], t);
                e[i] = ekp + re + t;
            } else {
                s[i] = kp + rs;
            }
        }
    }
}

// Inverse of reduce_scatter's distribution: every lane of the segment ends
// with all V values (own NV values start in a[0..NV-1]).
template <int LPC, int V, typename R>
__device__ __forceinline__ void all_gather(R (&a)[V], int lane)
{
    constexpr int LS = LPC < V ? LPC : V;
    constexpr int NV0 = V / LS;
#pragma unroll
    for (int o = 1; o < LS; o <<= 1) {
        const int n = NV0 * o;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const R rv = __shfl_xor_sync(FULL, a[i], o);
            const R lo = up ? rv : a[i];
            const R hi = up ? a[i] : rv;
            a[i] = lo;
            a[n + i] = hi;
        }
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Sum (a, b) over the block in a fixed order; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &b)
{
    __shared__ double sh[2][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; }
    __syncthreads();
    if (warp == 0) {
        a = lane < nw ? sh[0][lane] : 0.0;
        b = lane < nw ? sh[1][lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
    __syncthreads();
}

// Last-block finalisation of one iteration: sum the per-block partials in a
// fixed order, form the relative change of phi, update the state and the
// graph's loop condition.
// phase 0: the plain iteration; 1: an iteration that leaves its halo in BF16
// (never final: ends the BF16 phase with ST_SWITCH instead of converging);
// 3: the iteration back to FP32 after ST_SWITCH (never final either); 4: the
// correction iteration of the FP32 refinement.  Its scalar flux comes from the
// incident correction alone, which is zero in its first iteration, so the
// relative change of that iteration says nothing: it never converges there;
// and it has no stall stop (it runs to tol or max_iter).
__device__ __forceinline__ void finalize_iteration(double d2, double p2, double *partials, IterState *st,
                                                   const IterConfig *cfg, int iter, int use_cond,
                                                   cudaGraphConditionalHandle cond, int phase = 0)
{
    __shared__ int is_last;
    block_sum2(d2, p2);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = d2;
        partials[2 * blockIdx.x + 1] = p2;
        __threadfence();
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        a += __ldcg(partials + 2 * i);
        b += __ldcg(partials + 2 * i + 1);
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        const int it = iter + 1;
        double resid;
        if (b > 0.0) resid = sqrt(a / b);
        else resid = (a == 0.0) ? 0.0 : __longlong_as_double(0x7ff0000000000000LL);
        st->iter = it;
        st->resid = resid;
        st->d2 = a;
        st->p2 = b;
        st->arrive = 0u;
        if ((phase == 1 || phase == 3) && (st->status == ST_RUNNING || (phase == 3 && st->status == ST_SWITCH))) {
            int ns = ST_RUNNING;
            if (!(resid == resid) || !(a == a) || !(b == b) || isinf(b)) ns = ST_NAN;
            else if (phase == 1 && (resid < cfg->halo_switch || it >= cfg->max_iter - 2)) ns = ST_SWITCH;
            if (phase == 3) {  // the FP32 iterations start their stall tracking afresh
                st->stall = 0;
                st->best = __longlong_as_double(0x7ff0000000000000LL);
            }
            st->status = ns;
        } else if ((phase == 0 || phase == 4) && st->status == ST_RUNNING) {
            int ns = ST_RUNNING;
            if (!(resid == resid) || !(a == a) || !(b == b) || isinf(b)) ns = ST_NAN;
            else if (resid < cfg->tol && (phase == 0 || it > st->lin_first)) ns = ST_CONVERGED;
            else if (it >= cfg->max_iter) ns = ST_MAXITER;
            if (ns == ST_RUNNING && phase == 0 && cfg->stall_floor > 0.0) {
                // rounding-noise floor: the change stopped falling well above tol
                // (stall_iters < 0: stop as soon as it is below stall_floor)
                if (cfg->stall_iters < 0) {
                    if (resid < cfg->stall_floor) ns = ST_STALL;
                } else if (resid < 0.9 * st->best) {
                    st->best = resid;
                    st->stall = 0;
                } else if (++st->stall >= cfg->stall_iters && resid < cfg->stall_floor) {
                    ns = ST_STALL;
                }
            }
            st->status = ns;
            const bool go_on = ns == ST_RUNNING && it != cfg->pause_at;  // pause: host resumes the step
            if (use_cond) cudaGraphSetConditional(cond, go_on ? 1u : 0u);
        } else if (use_cond) {
            // stopped during this launch (guard or copy timeout): end the loop
            cudaGraphSetConditional(cond, 0u);
        }
    }
}

// Iteration prologue shared by the iteration kernels: read the state, trip
// the launch guard, stop the loop when the step is already decided.
// Returns false when the kernel has nothing to do.
template <typename R>
__device__ __forceinline__ bool iteration_prologue(const KParams<R> &p, int &iter, int &base, bool after_switch = false)
{
    IterState *st = p.st;
    const int status = *(volatile int *)&st->status;
    iter = *(volatile int *)&st->iter;
    base = *(volatile int *)&st->base;
    if (after_switch) return status == ST_SWITCH;  // the one iteration back to FP32 faces
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // launches while running (a graph body may hold several launches; those
        // after the step ended return at once and are not counted)
        const int launches = status == ST_RUNNING ? atomicAdd(&st->launches, 1) : 0;
        if (status == ST_RUNNING && launches >= p.cfg->max_iter + 2) {
            // The loop should have ended: report; this launch's last block
            // ends the loop.
            st->status = ST_GUARD;
        } else if (status != ST_RUNNING && p.use_cond) {
            cudaGraphSetConditional(p.cond, 0u);
        }
    }
    return status == ST_RUNNING;
}

// ---------------------------------------------------------------------------
// One iteration over all cells.
//   M_OCI: phi^{l+1} = K r with r = sum w A^{-1} c(halo^l); outgoing corners
//          y_out + s (A^{-1} phi)_out into the other face buffer.
//   M_SI : the scalar-flux update after a sweep: phi^{l+1} = sum w A^{-1}
//          (c(faces^{l+1}) + s phi^l), and the next sweep's affine offsets
//          g = (A^{-1}(c_fixed + s phi^{l+1}))_out.
// LPC lanes per cell (power of two <= 32), PPL pairs per lane, CHUNK cell rows
// per warp pass.
// ---------------------------------------------------------------------------
template <typename R, int LPC, int PPL, int CHUNK, int MODE>
__global__ void __launch_bounds__(256) k_cells(const KParams<R> p)
{
    constexpr int SPW = 32 / LPC;
    constexpr int CPC = CHUNK * SPW;
    constexpr int V = 4 * CHUNK;
    constexpr bool COMP = sizeof(R) == 4;
    constexpr int NV = (V >= LPC) ? V / LPC : 1;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int seg = lane / LPC, ls = lane % LPC;
    const int J = p.J, P = p.P;

    int iter, base;
    if (!iteration_prologue(p, iter, base)) return;
    const int frd = MODE == M_OCI ? ((base + iter) & 1) : base;
    const int fwr = frd ^ 1;
    const phi_t<R> *phr = iter == 0 ? p.phi0 : p.phi[iter & 1];
    phi_t<R> *phw = p.phi[(iter + 1) & 1];
    const r2<R> *fPr = p.faceP[frd], *fMr = p.faceM[frd];
    r2<R> *fPw = p.faceP[fwr], *fMw = p.faceM[fwr];
    const bool refl_l = MODE == M_OCI && p.bc_left == BC_REFLECT;
    const bool refl_r = MODE == M_OCI && p.bc_right == BC_REFLECT;

    double acc_d2 = 0.0, acc_p2 = 0.0;
    float accf_d2 = 0.f, accf_p2 = 0.f;  // FP32 mode: per-lane partials (grid sums in double)
    const int nchunks = (J + CPC - 1) / CPC;
    for (int chunk = blockIdx.x * wpb + warp; chunk < nchunks; chunk += gridDim.x * wpb) {
        R s_acc[V], e_acc[V];
        R yo[CHUNK][PPL][4];
        // ---------------- phase A: per-ordinate block solves y = A^{-1} c
#pragma unroll
        for (int r = 0; r < CHUNK; ++r) {
            const int cell = chunk * CPC + r * SPW + seg;
            const bool valid = cell < J;
            const int m = valid ? __ldg(p.mat + cell) : 0;
            const r4<R> qd = valid ? ldg4(p.cellq + cell) : r4<R>{0, 0, 0, 0};
            const r2<R> es = ldg2(p.matpar + m);
            R fkl = 0, fkr = 0, fhl = 0, fhr = 0;
            if (MODE == M_SI && valid) {
                load_phi4<R>(phr, cell, fkl, fkr, fhl, fhr);
                fkl *= es.y; fkr *= es.y; fhl *= es.y; fhr *= es.y;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) { s_acc[4 * r + k] = 0; e_acc[4 * r + k] = 0; }
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                const int pp = ls + LPC * i;
                yo[r][i][0] = yo[r][i][1] = yo[r][i][2] = yo[r][i][3] = 0;
                if (valid && pp < P) {
                    const Coef<R> a = load_coef(p.tab, m, P, pp);
                    const r2<R> mw = ldg2(p.muw + pp);
                    const r2<R> inP = (refl_l && cell == 0) ? ld2(fMr + pp) : ld2(fPr + (size_t)cell * P + pp);
                    const r2<R> inM = (refl_r && cell == J - 1) ? ld2(fPr + (size_t)J * P + pp)
                                                                : ld2(fMr + (size_t)(cell + 1) * P + pp);
                    const r4<R> pe = ld4(p.psi_edge + (size_t)cell * P + pp);
                    // fixed part of c (source + time edge), u+ = c+, u- = conj(c-)
                    R ukr = qd.x + es.x * pe.x, uki = qd.y + es.x * pe.y, uhr = qd.z, uhi = qd.w;
                    R vkr = qd.x + es.x * pe.z, vki = -(qd.y + es.x * pe.w), vhr = qd.z, vhi = -qd.w;
                    if (MODE == M_SI) {
                        // outgoing part of A^{-1} c_fixed (source and time edge only); the
                        // next sweep's offset adds s (A^{-1} phi^{l+1})_out after the update
                        yo[r][i][0] = a.pr * uki + a.pi * ukr + a.rr * uhi + a.ri * uhr;
                        yo[r][i][1] = a.ur * uki + a.ui * ukr + a.vr * uhi + a.vi * uhr;
                        yo[r][i][2] = a.pr * vkr - a.pi * vki + a.rr * vhr - a.ri * vhi;
                        yo[r][i][3] = a.ur * vkr - a.ui * vki + a.vr * vhr - a.vi * vhi;
                        // lagged scattering source s phi^l (b^+/b^- of the SI section)
                        ukr += fkl; uki += fkr; uhr += fhl; uhi += fhr;
                        vkr += fkl; vki -= fkr; vhr += fhl; vhi -= fhr;
                        if (cell == J - 1 && p.bc_right == BC_REFLECT)  // lag for the next sweep
                            st2(p.refl + pp, ld2(fPr + (size_t)J * P + pp).x, ld2(fPr + (size_t)J * P + pp).y);
                    }
                    // incident terms: +mu enters rows 1, 3 (corner L); -mu rows 2, 4 (corner R)
                    ukr += mw.x * inP.x; uhr += mw.x * inP.y;
                    vki -= mw.x * inM.x; vhi -= mw.x * inM.y;
                    R ykr, yki, yhr, yhi, zkr, zki, zhr, zhi;
                    ainv(a, ukr, uki, uhr, uhi, ykr, yki, yhr, yhi);
                    ainv(a, vkr, vki, vhr, vhi, zkr, zki, zhr, zhi);
                    if (MODE == M_OCI) {
                        yo[r][i][0] = yki; yo[r][i][1] = yhi; yo[r][i][2] = zkr; yo[r][i][3] = zhr;
                    }
                    // w (y+ + conj(z)): moments (kL, kR, hL, hR)
                    const R c0 = mw.y * (ykr + zkr), c1 = mw.y * (yki - zki);
                    const R c2 = mw.y * (yhr + zhr), c3 = mw.y * (yhi - zhi);
                    if (PPL == 1) {
                        s_acc[4 * r + 0] = c0; s_acc[4 * r + 1] = c1; s_acc[4 * r + 2] = c2; s_acc[4 * r + 3] = c3;
                    } else {
                        R t;
                        two_sum(s_acc[4 * r + 0], c0, s_acc[4 * r + 0], t); e_acc[4 * r + 0] += t;
                        two_sum(s_acc[4 * r + 1], c1, s_acc[4 * r + 1], t); e_acc[4 * r + 1] += t;
                        two_sum(s_acc[4 * r + 2], c2, s_acc[4 * r + 2], t); e_acc[4 * r + 2] += t;
                        two_sum(s_acc[4 * r + 3], c3, s_acc[4 * r + 3], t); e_acc[4 * r + 3] += t;
                    }
                }
            }
        }
        // ---------------- phase B: moments over the segment's lanes
        reduce_scatter<LPC, V, COMP>(s_acc, e_acc, lane);
        // ---------------- phase C: capacitance solve + residual, in double
        const int base_idx = (V >= LPC) ? NV * ls : (ls % V);
        const bool owner_lane = (V >= LPC) || (ls < V);
        R phiR[V];
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const int gi = base_idx + t;
            const int row = gi >> 2, comp = gi & 3;
            const int cell = chunk * CPC + row * SPW + seg;
            if constexpr (sizeof(R) == 4) {
                // FP32 mode: double-float capacitance solve and iterate difference
                const ff r_own = ff_norm(s_acc[t], e_acc[t]);
                ff phi;
                if (MODE == M_OCI) {
                    ff r_par;
                    if constexpr (NV >= 4) {
                        r_par = ff_norm(s_acc[t ^ 2], e_acc[t ^ 2]);
                    } else {
                        constexpr int o = NV == 2 ? 1 : 2;
                        r_par.h = __shfl_xor_sync(FULL, r_own.h, o);
                        r_par.l = __shfl_xor_sync(FULL, r_own.l, o);
                    }
                    const int m = cell < J ? __ldg(p.mat + cell) : 0;
                    const float4 k0 = __ldg(p.matKf + 2 * m), k1 = __ldg(p.matKf + 2 * m + 1);
                    phi = comp < 2 ? ff_add(ff_mul(ff{k0.x, k0.y}, r_own), ff_mul(ff{k0.z, k0.w}, r_par))
                                   : ff_add(ff_mul(ff{k1.x, k1.y}, r_par), ff_mul(ff{k1.z, k1.w}, r_own));
                } else {
                    phi = r_own;
                }
                if (owner_lane && cell < J) {
                    const float2 old = __ldcg(reinterpret_cast<const float2 *>(phr) + 4 * (size_t)cell + comp);
                    const float d = ff_diff(phi, ff{old.x, old.y});
                    accf_d2 = __fmaf_rn(d, d, accf_d2);
                    accf_p2 = __fmaf_rn(phi.h, phi.h, accf_p2);
                    reinterpret_cast<float2 *>(phw)[4 * (size_t)cell + comp] = make_float2(phi.h, phi.l);
                }
                phiR[t] = (R)__fadd_rn(phi.h, phi.l);
            } else {
                const double r_own = (double)s_acc[t] + (double)e_acc[t];
                double phi;
                if (MODE == M_OCI) {
                    double r_par;
                    if constexpr (NV >= 4) r_par = (double)s_acc[t ^ 2] + (double)e_acc[t ^ 2];
                    else if constexpr (NV == 2) r_par = __shfl_xor_sync(FULL, r_own, 1);
                    else r_par = __shfl_xor_sync(FULL, r_own, 2);
                    const int m = cell < J ? __ldg(p.mat + cell) : 0;
                    const kmat K = p.matK[m];
                    phi = comp < 2 ? K.k00 * r_own + K.k01 * r_par : K.k10 * r_par + K.k11 * r_own;
                } else {
                    phi = r_own;
                }
                if (owner_lane && cell < J) {
                    const double old = __ldcg(reinterpret_cast<const double *>(phr) + 4 * (size_t)cell + comp);
                    const double d = phi - old;
                    acc_d2 += d * d;
                    acc_p2 += phi * phi;
                    reinterpret_cast<double *>(phw)[4 * (size_t)cell + comp] = phi;
                }
                phiR[t] = (R)phi;
            }
        }
        // ---------------- phase D: every lane of the segment gets phi of its cells
        all_gather<LPC, V>(phiR, lane);
        // ---------------- phase E: back-substitution of the outgoing corners
#pragma unroll
        for (int r = 0; r < CHUNK; ++r) {
            const int cell = chunk * CPC + r * SPW + seg;
            if (cell >= J) continue;
            const int m = __ldg(p.mat + cell);
            const R s = ldg2(p.matpar + m).y;
            const R Fkl = phiR[4 * r] * s, Fkr = phiR[4 * r + 1] * s, Fhl = phiR[4 * r + 2] * s, Fhr = phiR[4 * r + 3] * s;
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                const int pp = ls + LPC * i;
                if (pp >= P) continue;
                const Coef<R> a = load_coef(p.tab, m, P, pp);
                // +mu: Im(A^{-1} Phi); -mu: Re(A^{-1} conj(Phi))
                const R ok = yo[r][i][0] + (a.pr * Fkr + a.pi * Fkl + a.rr * Fhr + a.ri * Fhl);
                const R oh = yo[r][i][1] + (a.ur * Fkr + a.ui * Fkl + a.vr * Fhr + a.vi * Fhl);
                const R mk = yo[r][i][2] + (a.pr * Fkl + a.pi * Fkr + a.rr * Fhl + a.ri * Fhr);
                const R mh = yo[r][i][3] + (a.ur * Fkl + a.ui * Fkr + a.vr * Fhl + a.vi * Fhr);
                if (MODE == M_OCI) {
                    st2(fPw + (size_t)(cell + 1) * P + pp, ok, oh);
                    st2(fMw + (size_t)cell * P + pp, mk, mh);
                } else {
                    st4(p.g + (size_t)pp * J + cell, ok, oh, mk, mh);
                }
            }
        }
    }
    finalize_iteration(acc_d2 + (double)accf_d2, acc_p2 + (double)accf_p2, p.partials, p.st, p.cfg, iter,
                       p.use_cond, p.cond);
}

// ---------------------------------------------------------------------------
// Staged variant of k_cells for the bandwidth-bound FP32 path: a persistent
// grid in which every warp streams its 8-row chunks through a STAGES-deep ring
// in shared memory.  One lane issues bulk asynchronous copies (TMA,
// cp.async.bulk) of the chunk's contiguous rows -- incident faces, time-edge
// flux, source moments, material ids -- completing on a per-stage mbarrier;
// the warp computes chunk i while chunks i+1 .. i+STAGES-1 are in flight.
// Launched as a programmatic dependent of the previous iteration (stream
// launches with programmatic serialisation, programmatic graph edges): the
// copies that do not change between iterations (time-edge flux, sources,
// materials) of the first chunks are issued before griddepcontrol.wait, the
// state and the incident faces only after it, and the kernel allows its own
// dependent to launch as soon as it has read the state.  Without a
// programmatic launch both instructions are no-ops.
// Every mbarrier wait is bounded: on expiry the kernel records ST_TIMEOUT,
// drains (again bounded) its own copies and finishes the iteration normally.
// ---------------------------------------------------------------------------
constexpr unsigned kWaitLimit = 1u << 22;
template <bool B> struct BoolTag { static constexpr bool value = B; };

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(a) : "memory");
    return v;
}
// Grid-wide barrier of the persistent loop (all blocks resident: cooperative
// launch).  The arrival counter starts at 0 for each launch; the k-th barrier
// waits until it reaches k * gridDim.x.  Thread 0 alone meets the grid (the
// block's own writes were ordered before it by a block barrier): release-
// arrive on count (fence, then the atomic), then poll (bounded) with acquire
// loads until target arrivals; false when the limit expired.  The acquire load that sees the target, followed by the
// caller's block barrier, orders the other blocks' released writes before
// every thread's later reads, so no fence follows it.
__device__ __forceinline__ bool grid_arrive_wait(unsigned *count, unsigned target, unsigned limit)
{
    __threadfence();
    atomicAdd(count, 1u);
    for (unsigned it = 0; it < limit; ++it) {
        if (ld_acquire_u32(count) >= target) return true;
        __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx_arrive(unsigned long long *bar, unsigned bytes)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; false when the limit expired.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(d),
        "l"(src), "r"(bytes), "r"(b)
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__host__ __device__ constexpr unsigned round16(unsigned b) { return (b + 15u) & ~15u; }
// Barrier region at the start of the dynamic shared memory, padded so that the
// rings after it (bulk-copy destinations, 16-byte loads) stay 128-byte aligned.
__host__ __device__ constexpr unsigned tma_bar_bytes(int stages, int warps)
{
    return ((unsigned)(8 * stages * warps) + 127u) & ~127u;
}

// u = c (fixed part + incident), the complex right-hand sides of one ordinate
// pair, from the staged operands (u+ = c+, u- = conj(c-)).
template <typename R>
struct PairRhs { R ukr, uki, uhr, uhi, vkr, vki, vhr, vhi; };

template <typename R>
__device__ __forceinline__ PairRhs<R> pair_rhs_fixed(const r4<R> &qd, R e, const r4<R> &pe)
{
    return {qd.x + e * pe.x, qd.y + e * pe.y, qd.z, qd.w, qd.x + e * pe.z, -(qd.y + e * pe.w), qd.z, -qd.w};
}

// Per-warp transpose buffer of the staged kernel: 32 lanes x 32 partial sums
// (8 rows x 4 moments), XOR-swizzled in 16-byte groups (with the lane's low and
// segment bits) so that the row-wise vector stores and the column-wise scalar
// loads are bank-conflict free.
constexpr unsigned kXposeBytes = 32u * 32u * 4u;
__device__ __forceinline__ int xpose_idx(int l, int v)
{
    return 32 * l + 4 * (((v >> 2) ^ l ^ (l >> 3)) & 7) + (v & 3);
}

// Decision of the persistent loops after iteration it (1-based) from the grid
// sums a = sum (dphi)^2, b = sum phi^2: the next state and the stall tracking.
// halo2: the BF16 phase (never final; ST_SWITCH instead).
__device__ __forceinline__ int loop_decision(double a, double b, bool fault, int it, int fixed_left, bool halo2,
                                             const IterConfig *cfg, int &stall, double &best, double &resid)
{
    if (b > 0.0) resid = sqrt(a / b);
    else resid = (a == 0.0) ? 0.0 : __longlong_as_double(0x7ff0000000000000LL);
    int ns = ST_RUNNING;
    if (fault) ns = ST_TIMEOUT;
    else if (!(resid == resid) || !(a == a) || !(b == b) || isinf(b)) ns = ST_NAN;
    else if (fixed_left > 0) ns = it >= fixed_left ? ST_MAXITER : ST_RUNNING;  // timing: a fixed count
    else if (halo2) {
        // BF16 phase: never final; ends at the switch threshold, near the
        // iteration limit, or once BF16 rounding stops the change falling
        if (resid < cfg->halo_switch || it >= cfg->max_iter - 2) ns = ST_SWITCH;
        else if (resid < 0.9 * best) {
            best = resid;
            stall = 0;
        } else if (++stall >= cfg->halo_stall) {
            ns = ST_SWITCH;
        }
    }
    else if (resid < cfg->tol) ns = ST_CONVERGED;
    else if (it >= cfg->max_iter) ns = ST_MAXITER;
    if (!halo2 && ns == ST_RUNNING && fixed_left == 0 && cfg->stall_floor > 0.0) {
        if (cfg->stall_iters < 0) {
            if (resid < cfg->stall_floor) ns = ST_STALL;
        } else if (resid < 0.9 * best) {
            best = resid;
            stall = 0;
        } else if (++stall >= cfg->stall_iters && resid < cfg->stall_floor) {
            ns = ST_STALL;
        }
    }
    return ns;
}

__device__ __forceinline__ void st_release_u32(unsigned *a, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *a)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(a) : "memory");
    return v;
}

template <typename R, int LPC, int PPL, int MODE>
__device__ __forceinline__ void percell_body(const KParams<R> &p, int gw, int nwarps, int frd, int fgs,
                                             const phi_t<R> *phi_psi, const phi_t<R> *phi_pub);

// HALO (OCI only) selects the storage of the face buffers the iteration reads
// and writes: 0 float pairs in and out; 1 float in, BF16 out (first iteration
// of the BF16 phase); 2 BF16 in and out (the phase's persistent loop); 3 BF16
// in, float out (the iteration back to FP32 after ST_SWITCH).
// Threads per block of the staged kernel: the rings of 8-row chunks fit 11
// warps in shared memory, those of 4-row chunks of one pair per lane 18 (at
// S_64 that layout measured 27 % slower per iteration than 8-row chunks with
// 11 warps: the warps' own instruction-level parallelism matters more).
__host__ __device__ constexpr int tma_max_threads(int chunk, int ppl) { return (chunk >= 8 || ppl > 1) ? 384 : 576; }

// ASYNC (persistent OCI loop, float faces): no grid barrier between
// iterations.  Block b owns a contiguous run of chunks; only its two edge
// chunks read faces another block writes.  Per iteration a block meets at one
// block barrier; its warp 0 then publishes the block's partial sums of the
// iteration just finished and a "finished" flag for the neighbouring blocks,
// and arrives at a counter; the last block to arrive adds every block's
// partial in a fixed order and publishes the decision (the same sums every
// run).  The other warps go straight on with the next iteration's interior
// chunks; an edge chunk waits for its neighbouring block's flag.  An
// iteration may so start before the previous one is decided: the faces
// rotate through three buffers, so that speculative iteration overwrites
// neither the decided iteration's input faces nor its moments; it stops at the
// first chunk boundary after the decision is seen, and no iteration starts
// writing before the decision of the one two back is known.  The end of the
// step (commit) follows one grid barrier.
template <int LPC, int PPL, int CHUNK, int STAGES, int MODE, bool LOOP = false, int HALO = 0, bool ASYNC = false>
__global__ void __launch_bounds__(tma_max_threads(CHUNK, PPL), 1) k_cells_tma(const KParams<float> p)
{
    using R = float;
    constexpr int SPW = 32 / LPC;
    constexpr int CPC = CHUNK * SPW;
    constexpr int V = 4 * CHUNK;           // partial sums per lane
    constexpr int NOWN = (V * SPW) / 32 > 0 ? (V * SPW) / 32 : 1;  // (segment, value) sums owned per lane
    static_assert(!LOOP || MODE == M_OCI, "the persistent loop runs the OCI iteration only");
    static_assert(HALO == 0 || MODE == M_OCI, "BF16 faces in the OCI iteration only");
    static_assert(!LOOP || HALO == 0 || HALO == 2, "the persistent loops keep one face storage");
    static_assert(!ASYNC || (LOOP && HALO == 0), "the barrier-free loop is the float-face OCI loop");
    constexpr bool IN_BF = HALO == 2 || HALO == 3, OUT_BF = HALO == 1 || HALO == 2;
    constexpr unsigned FB = IN_BF ? 4u : 8u;  // bytes per face pair read
    extern __shared__ __align__(128) unsigned char smem[];
    // a step held by its prologue (queued behind a step that did not commit):
    // every block leaves before touching anything
    if (LOOP && __ldcg(&p.st->status) == ST_HELD) return;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int seg = lane / LPC, ls = lane % LPC;
    const int J = p.J, P = p.P;

    constexpr bool PING = MODE == M_OCI || MODE == M_LIN;  // iterate in the face buffers
    const r4<R> *edge_src = MODE == M_LIN ? p.r0 : p.psi_edge;
    // shared memory: [barriers][per-warp transpose buffers][per-warp rings]
    const unsigned oP = 0, oM = round16(CPC * P * 8u), oE = 2 * round16(CPC * P * 8u);
    const unsigned oQ = oE + round16(CPC * P * 16u), oT = oQ + round16(CPC * 16u);
    const unsigned sbytes = oT + round16(CPC * 4u);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem) + warp * STAGES;
    float *xp = reinterpret_cast<float *>(smem + tma_bar_bytes(STAGES, wpb) + (size_t)warp * kXposeBytes);
    unsigned char *ring = smem + tma_bar_bytes(STAGES, wpb) + (size_t)wpb * kXposeBytes + (size_t)warp * STAGES * sbytes;
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(bars + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    fence_proxy_async();
    __syncwarp();

    const int nchunks = (J + CPC - 1) / CPC;
    const int gw = blockIdx.x * wpb + warp, tw = gridDim.x * wpb;
    // Chunk ownership.  Barrier loop: chunk gw + i tw (round robin over every
    // warp of the grid).  ASYNC: block b owns the contiguous chunks [cb0, cb1),
    // its warps take them round robin, and warp 0 takes its first chunk (the
    // block's left edge) last, so that both edge chunks -- the only ones that
    // read faces written by another block -- come at the end of an iteration.
    const int cb0 = ASYNC ? (int)(((long long)blockIdx.x * nchunks) / gridDim.x) : 0;
    const int cb1 = ASYNC ? (int)(((long long)(blockIdx.x + 1) * nchunks) / gridDim.x) : 0;
    const int nmine = ASYNC ? (warp < cb1 - cb0 ? (cb1 - cb0 - 1 - warp) / wpb + 1 : 0)
                            : (gw < nchunks ? (nchunks - 1 - gw) / tw + 1 : 0);
    auto chunk_of = [&](int i) -> int {
        if constexpr (ASYNC) return cb0 + warp + ((warp == 0 && nmine > 1) ? (i + 1) % nmine : i) * wpb;
        else return gw + i * tw;
    };
    // ring position of this iteration's local chunk 0 (the ring runs on across
    // the iterations of the persistent loop): local chunk i uses stage
    // (rp + i) % STAGES with phase parity ((rp + i) / STAGES) & 1
    int rp = 0;
    auto stage_of = [&](int i) { return (rp + i) % STAGES; };
    auto parity_of = [&](int i) { return (unsigned)((rp + i) / STAGES) & 1u; };

    auto issue_static = [&](int i) {  // lane 0: iteration-invariant copies of local chunk i
        if (i >= nmine) return;
        const int c0 = chunk_of(i) * CPC;
        const int nv = J - c0 < CPC ? J - c0 : CPC;
        unsigned char *st = ring + (size_t)stage_of(i) * sbytes;
        unsigned long long *bar = bars + stage_of(i);
        const unsigned bE = round16(nv * P * 16u), bQ = nv * 16u, bT = round16(nv * 4u);
        mbar_expect_tx(bar, bE + bQ + bT);
        bulk_g2s(st + oE, edge_src + (size_t)c0 * P, bE, bar);
        bulk_g2s(st + oQ, p.cellq + c0, bQ, bar);
        bulk_g2s(st + oT, p.mat + c0, bT, bar);
    };
    // complete the phases of copies issued for chunks that will not run (the
    // ASYNC loop issues every copy of a chunk at once, none ahead of its iteration)
    auto drain_static = [&]() {
        if constexpr (!ASYNC) {
            if (lane == 0)
                for (int i = 0; i < STAGES - 1 && i < nmine; ++i) mbar_arrive(bars + stage_of(i));
            for (int i = 0; i < STAGES - 1 && i < nmine; ++i) (void)mbar_wait(bars + stage_of(i), parity_of(i));
        }
    };
    if (!ASYNC && lane == 0)
        for (int i = 0; i < STAGES - 1; ++i) issue_static(i);
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    int iter, base;
    // persistent loop: the step state is kept by every block (all take the same
    // decisions from the same per-block partial sums); block 0 publishes it
    int status = ST_RUNNING, stall = 0, fixed_left = 0;
    double best = 0.0;
    if constexpr (LOOP) {
        const IterState *st0 = p.st;
        status = *(volatile const int *)&st0->status;
        iter = *(volatile const int *)&st0->iter;
        base = *(volatile const int *)&st0->base;
        stall = *(volatile const int *)&st0->stall;
        best = *(volatile const double *)&st0->best;
        fixed_left = p.loop_fixed;
        if (status != ST_RUNNING) {
            drain_static();
            return;
        }
    } else {
        if (!iteration_prologue(p, iter, base, HALO == 3)) {
            drain_static();
            return;
        }
    }
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const bool refl_l = PING && p.bc_left == BC_REFLECT;
    const bool refl_r = PING && p.bc_right == BC_REFLECT;

    // pair constants and a per-lane cache of the material coefficients
    r2<R> mw[PPL];
#pragma unroll
    for (int t = 0; t < PPL; ++t) mw[t] = (ls + LPC * t < P) ? ldg2(p.muw + ls + LPC * t) : r2<R>{0, 0};
    int mc = -1;
    Coef<R> ac[PPL];
    R ce = 0, cs = 0;
    auto coefs = [&](int m) {
        if (m != mc) {
            mc = m;
            const r2<R> es = ldg2(p.matpar + m);
            ce = es.x;
            cs = es.y;
#pragma unroll
            for (int t = 0; t < PPL; ++t) {
                const int pp = ls + LPC * t;
                if (pp < P) ac[t] = load_coef(p.tab, m, P, pp);
            }
        }
    };
    int mK = -1;
    float4 kA = make_float4(0.f, 0.f, 0.f, 0.f), kB = kA;
    // ASYNC: the blocks owning the chunks next to this block's edges (-1: none;
    // block b owns [floor(b n / G), floor((b + 1) n / G)), so chunk c belongs to
    // block floor(((c + 1) G - 1) / n)), wait limit, the launch's starting stall state
    auto chunk_owner = [&](int c) { return (int)((((long long)c + 1) * gridDim.x - 1) / nchunks); };
    const int nb_left = (ASYNC && cb1 > cb0 && cb0 > 0) ? chunk_owner(cb0 - 1) : -1;
    const int nb_right = (ASYNC && cb1 > cb0 && cb1 < nchunks) ? chunk_owner(cb1) : -1;
    const unsigned shortfall = LOOP ? (unsigned)p.cfg->bar_shortfall : 0u;
    const unsigned wlimit = LOOP && p.cfg->bar_poll_limit ? p.cfg->bar_poll_limit : kWaitLimit;
    const int stall0 = stall;
    const double best0 = best;
    // ASYNC: per-warp partials of the last two iterations, and the block's stop flag
    // (set by any warp that saw the step end; read by all after a block barrier)
    __shared__ double s_wpart[ASYNC ? 2 : 1][ASYNC ? tma_max_threads(CHUNK, PPL) / 32 : 1][3];
    // (two slots by iteration parity: iteration r sets slot r & 1, read by every
    // thread after the block barrier at the top of iteration r + 1, while the
    // first warps already running r + 1 may set the other slot)
    __shared__ int s_stop[2];
    if constexpr (ASYNC) {
        if (threadIdx.x < 2) s_stop[threadIdx.x] = 0;
        __syncthreads();
    }
    // ASYNC, lane 0: bounded wait for the decision of iteration q of this launch;
    // 1 the step goes on, 2 it ended there, 0 the wait ran out
    auto wait_decision = [&](int q) -> int {
        for (unsigned it = 0; it < wlimit; ++it) {
            if (ld_acquire_u32(&p.as->tag[q & 3]) == (unsigned)q + 1u)
                return *(volatile const int *)&p.as->rec[q & 3].status == ST_RUNNING ? 1 : 2;
            __nanosleep(20);
        }
        return 0;
    };

    // End of a step inside the persistent loops (multiple balance: psi_{k+1/2} of
    // every ordinate and corner, A^{-1}(c + s phi) with the incident faces the last
    // iteration read (buffer frd_l), becomes psi_edge; its outgoing corners, in
    // buffer fgs, are the next step's initial iterate; phi is published).  Each
    // warp streams its own chunks through its ring, so the pass runs at an
    // iteration's memory-level parallelism.  It starts at ring position rp with
    // no copy in flight; it writes psi_edge of its own cells and buffer fgs.
    auto ring_commit = [&](int frd_l, int fgs, const phi_t<R> *phf) {
        const bool ext = p.cfg->extrap != 0;
        auto issue_commit = [&](int i) {  // lane 0: every copy of local chunk i
            if (i >= nmine) return;
            const int c0 = chunk_of(i) * CPC;
            const int nv = J - c0 < CPC ? J - c0 : CPC;
            unsigned char *stg = ring + (size_t)stage_of(i) * sbytes;
            unsigned long long *bar = bars + stage_of(i);
            const unsigned bF = round16(nv * P * 8u), bE = round16(nv * P * 16u), bQ = nv * 16u,
                           bT = round16(nv * 4u);
            mbar_expect_tx_arrive(bar, 2 * bF + bE + bQ + bT);
            bulk_g2s(stg + oP, p.faceP[frd_l] + (size_t)c0 * P, bF, bar);
            bulk_g2s(stg + oM, p.faceM[frd_l] + (size_t)(c0 + 1) * P, bF, bar);
            bulk_g2s(stg + oE, p.psi_edge + (size_t)c0 * P, bE, bar);
            bulk_g2s(stg + oQ, p.cellq + c0, bQ, bar);
            bulk_g2s(stg + oT, p.mat + c0, bT, bar);
        };
        if (lane == 0) {
            asm volatile("fence.proxy.async.global;\n" ::: "memory");
            for (int i = 0; i < STAGES - 1; ++i) issue_commit(i);
        }
        int broke = nmine;
        for (int i = 0; i < nmine; ++i) {
            if (lane == 0) {
                fence_proxy_async();
                issue_commit(i + STAGES - 1);
            }
            const int chunk = chunk_of(i);
            // this lane's rows' moments, loaded before the wait
            float2 fph[CHUNK][4];
#pragma unroll
            for (int r = 0; r < CHUNK; ++r) {
                const int cell = chunk * CPC + r * SPW + seg;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    fph[r][c] = cell < J ? __ldcg(phf + 4 * (size_t)cell + c) : make_float2(0.f, 0.f);
            }
            if (!mbar_wait(bars + stage_of(i), parity_of(i))) {
                broke = i;
                break;
            }
            const unsigned char *stg = ring + (size_t)stage_of(i) * sbytes;
            const r2<R> *sP = reinterpret_cast<const r2<R> *>(stg + oP);
            const r2<R> *sM = reinterpret_cast<const r2<R> *>(stg + oM);
            const r4<R> *sE = reinterpret_cast<const r4<R> *>(stg + oE);
            const r4<R> *sQ = reinterpret_cast<const r4<R> *>(stg + oQ);
            const int *sT = reinterpret_cast<const int *>(stg + oT);
#pragma unroll
            for (int r = 0; r < CHUNK; ++r) {
                const int cl = r * SPW + seg;
                const int cell = chunk * CPC + cl;
                if (cell >= J) continue;
                coefs(sT[cl]);
                const r4<R> qd = sQ[cl];
                const R Fkl = PhiStore<R>::real(fph[r][0]) * cs, Fkr = PhiStore<R>::real(fph[r][1]) * cs,
                        Fhl = PhiStore<R>::real(fph[r][2]) * cs, Fhr = PhiStore<R>::real(fph[r][3]) * cs;
#pragma unroll
                for (int t = 0; t < PPL; ++t) {
                    const int pp = ls + LPC * t;
                    if (pp >= P) continue;
                    const Coef<R> &a = ac[t];
                    const r4<R> pe = sE[cl * P + pp];
                    const r2<R> inP = (refl_l && cell == 0) ? ldcg2(p.faceM[frd_l] + pp) : sP[cl * P + pp];
                    const r2<R> inM = (refl_r && cell == J - 1) ? ldcg2(p.faceP[frd_l] + (size_t)J * P + pp)
                                                                : sM[cl * P + pp];
                    // end-of-step components (k+1/2): second rows of A^{-1}
                    R phr_, phi_, mhr, mhi;
                    commit_corners<R>(a, qd, ce, pe, Fkl, Fkr, Fhl, Fhr, mw[t].x, inP, inM, phr_, phi_, mhr, mhi);
                    st4(p.psi_edge + (size_t)cell * P + pp, phr_, phi_, mhr, -mhi);
                    if (ext) {  // linear in time through the previous end-of-step flux pe
                        const R dP = phi_ - pe.y, dM = mhr - pe.z;
                        st2(p.faceP[fgs] + (size_t)(cell + 1) * P + pp, phi_ + R(0.5) * dP, phi_ + dP);
                        st2(p.faceM[fgs] + (size_t)cell * P + pp, mhr + R(0.5) * dM, mhr + dM);
                    } else {
                        st2(p.faceP[fgs] + (size_t)(cell + 1) * P + pp, phi_, phi_);
                        st2(p.faceM[fgs] + (size_t)cell * P + pp, mhr, mhr);
                    }
                }
                for (int c = ls; c < 4; c += LPC) {
                    const float2 v = c == 0 ? fph[r][0] : c == 1 ? fph[r][1] : c == 2 ? fph[r][2] : fph[r][3];
                    p.phi_out[4 * (size_t)cell + c] = PhiStore<R>::wide(v);
                    p.phi0[4 * (size_t)cell + c] = (c & 1) ? fph[r][3] : fph[r][2];
                }
            }
            fence_proxy_async();
            __syncwarp();  // stage i fully read before a copy reuses it
        }
        if (broke < nmine) {
            // a copy never completed: record it and wait (bounded) for this warp's
            // outstanding copies before the shared memory goes
            if (lane == 0) atomicExch(&p.st->status, ST_TIMEOUT);
            const int last = broke + STAGES - 1 < nmine ? broke + STAGES - 1 : nmine - 1;
            for (int k = broke; k <= last; ++k) (void)mbar_wait(bars + stage_of(k), parity_of(k));
        } else {
            rp += nmine;
        }
    };

    for (int rep = 0;; ++rep) {
        const int frd = ASYNC ? (base + iter) % 3 : (PING ? ((base + iter) & 1) : base);
        const int fwr = ASYNC ? (base + iter + 1) % 3 : frd ^ 1;
        const phi_t<R> *phr = iter == 0 ? p.phi0 : p.phi[iter & 1];
        phi_t<R> *phw = p.phi[(iter + 1) & 1];
        const r2<R> *fPr = p.faceP[frd], *fMr = p.faceM[frd];
        r2<R> *fPw = p.faceP[fwr], *fMw = p.faceM[fwr];
        const unsigned *hPr = p.hfP[frd & 1], *hMr = p.hfM[frd & 1];  // BF16 phases use parities 0 and 1 only
        unsigned *hPw = p.hfP[fwr & 1], *hMw = p.hfM[fwr & 1];
        // incident faces at face index f: the staged copy's source, a boundary read
        auto face_src_P = [&](size_t f) -> const void * { return IN_BF ? (const void *)(hPr + f * P) : (const void *)(fPr + f * P); };
        auto face_src_M = [&](size_t f) -> const void * { return IN_BF ? (const void *)(hMr + f * P) : (const void *)(fMr + f * P); };
        auto face_ld_P = [&](size_t i) -> r2<R> {
            if constexpr (IN_BF) return unpack_bf16x2(hPr[i]);
            else return ld2(fPr + i);
        };
        auto face_ld_M = [&](size_t i) -> r2<R> {
            if constexpr (IN_BF) return unpack_bf16x2(hMr[i]);
            else return ld2(fMr + i);
        };

        auto issue_faces = [&](int i) {  // lane 0: this iteration's incident faces of local chunk i
            if (i >= nmine) return;
            const int c0 = chunk_of(i) * CPC;
            const int nv = J - c0 < CPC ? J - c0 : CPC;
            unsigned char *st = ring + (size_t)stage_of(i) * sbytes;
            unsigned long long *bar = bars + stage_of(i);
            const unsigned bF = round16(nv * P * FB);
            mbar_expect_tx_arrive(bar, 2 * bF);
            bulk_g2s(st + oP, face_src_P((size_t)c0), bF, bar);
            bulk_g2s(st + oM, face_src_M((size_t)c0 + 1), bF, bar);
        };
        auto issue = [&](int i) {  // lane 0: all copies of local chunk i
            if (i >= nmine) return;
            if constexpr (ASYNC) {
                // an edge chunk reads faces the neighbouring block wrote in the
                // previous iteration: wait (bounded) until that block published it
                const int c = chunk_of(i);
                if (rep > 0 && ((c == cb0 && nb_left >= 0) || (c == cb1 - 1 && nb_right >= 0))) {
                    // A neighbour that stopped does not publish: it stopped because the
                    // decision of iteration rep - 2 ended the step, which ends this one too.
                    int ok = 1;
                    for (int s = 0; s < 2 && ok == 1; ++s) {
                        const int nb = s == 0 ? (c == cb0 ? nb_left : -1) : (c == cb1 - 1 ? nb_right : -1);
                        if (nb < 0) continue;
                        for (unsigned it = 0; ld_acquire_u32(p.as_done + nb) < (unsigned)rep; ++it) {
                            if (it >= wlimit) { ok = 0; break; }
                            if (rep >= 2 && ld_acquire_u32(&p.as->tag[(rep - 2) & 3]) == (unsigned)rep - 1u &&
                                *(volatile const int *)&p.as->rec[(rep - 2) & 3].status != ST_RUNNING) { ok = 2; break; }
                            __nanosleep(20);
                        }
                    }
                    if (ok != 1) {
                        if (ok == 0) atomicExch(&p.st->status, ST_TIMEOUT);
                        s_stop[rep & 1] = 1;
                    }
                    asm volatile("fence.proxy.async.global;\n" ::: "memory");
                }
            }
            const int c0 = chunk_of(i) * CPC;
            const int nv = J - c0 < CPC ? J - c0 : CPC;
            unsigned char *st = ring + (size_t)stage_of(i) * sbytes;
            unsigned long long *bar = bars + stage_of(i);
            const unsigned bF = round16(nv * P * FB), bE = round16(nv * P * 16u), bQ = nv * 16u,
                           bT = round16(nv * 4u);
            mbar_expect_tx_arrive(bar, 2 * bF + bE + bQ + bT);
            bulk_g2s(st + oP, face_src_P((size_t)c0), bF, bar);
            bulk_g2s(st + oM, face_src_M((size_t)c0 + 1), bF, bar);
            bulk_g2s(st + oE, edge_src + (size_t)c0 * P, bE, bar);
            bulk_g2s(st + oQ, p.cellq + c0, bQ, bar);
            bulk_g2s(st + oT, p.mat + c0, bT, bar);
        };
        if constexpr (ASYNC) {
            if (rep > 0) {
                __syncthreads();  // every warp of the block finished (or gave up) iteration rep - 1
                if (s_stop[(rep - 1) & 1]) break;
                // the block's generic face stores of rep - 1 made visible at device
                // scope (thread 0's fence covers every warp's, ordered by the block
                // barrier) before any warp's bulk copy reads them
                if (threadIdx.x == 0) __threadfence();
                __syncthreads();
                if (warp == 0) {
                    // publish iteration q = rep - 1: the block's partial (its warps' in
                    // a fixed order), then "finished q" for the neighbouring blocks,
                    // then the arrival; the last block to arrive sums every block's
                    // partial in a fixed order and publishes the decision
                    const int q = rep - 1;
                    int closer = 0;
                    if (lane == 0) {
                        double a = 0.0, b = 0.0, f = 0.0;
                        for (int w = 0; w < wpb; ++w) {
                            a += s_wpart[q & 1][w][0];
                            b += s_wpart[q & 1][w][1];
                            f += s_wpart[q & 1][w][2];
                        }
                        double *pp = p.as_part + ((size_t)(q & 3) * gridDim.x + blockIdx.x) * 3;
                        pp[0] = a;
                        pp[1] = b;
                        pp[2] = f;
                        // the block's faces and moments of q (ordered before this thread by
                        // the block barrier) and the partial, before the flag and the count
                        __threadfence();
                        st_release_u32(p.as_done + blockIdx.x, (unsigned)rep);
                        const unsigned old = atomicAdd(&p.as->cnt[q & 3], 1u);
                        closer = old + 1u == (unsigned)((q >> 2) + 1) * gridDim.x + shortfall ? 1 : 0;
                    }
                    closer = __shfl_sync(FULL, closer, 0);
                    if (closer) {
                        __threadfence();
                        const double *pp = p.as_part + (size_t)(q & 3) * gridDim.x * 3;
                        double a = 0.0, b = 0.0, f = 0.0;
                        for (int k = lane; k < (int)gridDim.x; k += 32) {
                            a += __ldcg(pp + 3 * k);
                            b += __ldcg(pp + 3 * k + 1);
                            f += __ldcg(pp + 3 * k + 2);
                        }
                        a = warp_sum(a);
                        b = warp_sum(b);
                        f = warp_sum(f);
                        if (lane == 0) {
                            int pstall = stall0, pstatus = ST_RUNNING;
                            double pbest = best0;
                            bool okq = true;
                            if (q > 0) {
                                // the previous decision's state (published before every
                                // block could arrive for q; waited for all the same)
                                okq = wait_decision(q - 1) != 0;
                                const AsyncRec *pr = &p.as->rec[(q - 1) & 3];
                                pstall = *(volatile const int *)&pr->stall;
                                pbest = *(volatile const double *)&pr->best;
                                pstatus = *(volatile const int *)&pr->status;
                            }
                            AsyncRec *rc = &p.as->rec[q & 3];
                            if (okq && pstatus != ST_RUNNING) {
                                // every block finished a speculative iteration after the
                                // step had ended: keep the earlier decision
                                rc->status = pstatus;
                                rc->stall = pstall;
                                rc->best = pbest;
                            } else {
                                const int it = iter;  // 1-based number of iteration q
                                double resid;
                                const int ns = loop_decision(a, b, f != 0.0 || !okq, it, fixed_left, false, p.cfg,
                                                             pstall, pbest, resid);
                                rc->resid = resid;
                                rc->d2 = a;
                                rc->p2 = b;
                                rc->best = pbest;
                                rc->stall = pstall;
                                rc->status = ns;
                                IterState *sw = p.st;
                                sw->iter = it;
                                sw->resid = resid;
                                sw->d2 = a;
                                sw->p2 = b;
                                sw->stall = pstall;
                                sw->best = pbest;
                                sw->launches += 1;
                                atomicCAS(&sw->status, ST_RUNNING, ns);  // a recorded timeout stays
                            }
                            __threadfence();
                            st_release_u32(&p.as->tag[q & 3], (unsigned)q + 1u);
                        }
                    }
                }
                // the block's own faces of rep - 1 (ordered by the block barrier)
                // before this warp's bulk reads of them
                if (lane == 0) asm volatile("fence.proxy.async.global;\n" ::: "memory");
            }
            // every copy of the first chunks of this iteration (an edge chunk waits
            // for its neighbouring block inside issue)
            if (lane == 0)
                for (int i = 0; i < STAGES - 1; ++i) issue(i);
        } else {
            // (in the barrier loop the first chunks' faces of iterations after the
            // first were issued right after the previous grid barrier)
            if (lane == 0 && !(LOOP && rep > 0))
                for (int i = 0; i < STAGES - 1; ++i) issue_faces(i);
        }
        // ASYNC: positions of the ring this iteration used; the decision of
        // iteration rep - 1, polled once per chunk (the load's latency hidden by
        // the chunk's work), ends a speculative iteration early
        int consumed = nmine;
        bool prev_known = !ASYNC || rep == 0;
        bool skip = false;
        if constexpr (ASYNC) {
            if (rep >= 2) {
                // this iteration overwrites the faces and moments iteration rep - 2
                // read: its decision must be known (and not final) first
                int go = 1;
                if (lane == 0) go = wait_decision(rep - 2);
                go = __shfl_sync(FULL, go, 0);
                if (go != 1) {
                    if (lane == 0) {
                        if (go == 0) atomicExch(&p.st->status, ST_TIMEOUT);
                        s_stop[rep & 1] = 1;
                    }
                    consumed = STAGES - 1 < nmine ? STAGES - 1 : nmine;
                    for (int k = 0; k < consumed; ++k) (void)mbar_wait(bars + stage_of(k), parity_of(k));
                    skip = true;
                }
            }
        }

        float accf_d2 = 0.f, accf_p2 = 0.f;  // per-lane partials; block and grid sums in double
        bool ok_all = true;
        int broke_at = nmine;
        for (int i = 0; i < (skip ? 0 : nmine); ++i) {
            if (lane == 0) {
                fence_proxy_async();
                issue(i + STAGES - 1);
            }
            unsigned poll_tag = 0;
            if (ASYNC && !prev_known && lane == 0 && i + 1 < nmine) poll_tag = ld_relaxed_u32(&p.as->tag[(rep - 1) & 3]);
            const int chunk = chunk_of(i);
            const unsigned char *st = ring + (size_t)stage_of(i) * sbytes;
            if (!mbar_wait(bars + stage_of(i), parity_of(i))) {
                ok_all = false;
                broke_at = i;
                break;
            }
            const r2<R> *sP = reinterpret_cast<const r2<R> *>(st + oP);
            const r2<R> *sM = reinterpret_cast<const r2<R> *>(st + oM);
            const unsigned *hsP = reinterpret_cast<const unsigned *>(st + oP);
            const unsigned *hsM = reinterpret_cast<const unsigned *>(st + oM);
            const r4<R> *sE = reinterpret_cast<const r4<R> *>(st + oE);
            const r4<R> *sQ = reinterpret_cast<const r4<R> *>(st + oQ);
            const int *sT = reinterpret_cast<const int *>(st + oT);
            // phi^l of the values this lane owns in phase C, fetched now so the
            // load overlaps phases A and B
            float2 old_phi[NOWN], ref_phi[NOWN];
    #pragma unroll
            for (int k = 0; k < NOWN; ++k) {
                const int f = lane * NOWN + k;
                const int g = f / V, v = f % V;
                const int cell = chunk * CPC + (v >> 2) * SPW + g;
                const bool ok = g < SPW && cell < J;
                old_phi[k] = ok ? __ldcg(phr + 4 * (size_t)cell + (v & 3)) : make_float2(0.f, 0.f);
                ref_phi[k] = (MODE == M_LIN && ok) ? __ldg(p.phi_ref + 4 * (size_t)cell + (v & 3)) : make_float2(0.f, 0.f);
            }
            // interior chunk of one material (no boundary cell, all rows present):
            // the per-row checks and coefficient lookups are hoisted
            const bool fast = chunk > 0 && (chunk + 1) * CPC < J && __all_sync(FULL, sT[lane % CPC] == sT[0]);
            if (fast) coefs(sT[0]);
            // ---------------- phase A: y = A^{-1} c per ordinate pair; lane partials
            // of the moments w (y+ + conj(y-)) go to the transpose buffer
            auto phase_a = [&](auto fast_tag) {
            constexpr bool FAST = decltype(fast_tag)::value;
    #pragma unroll
            for (int r = 0; r < CHUNK; ++r) {
                const int cl = r * SPW + seg;
                const int cell = chunk * CPC + cl;
                R m0 = 0, m1 = 0, m2 = 0, m3 = 0;
                if (FAST || cell < J) {
                    if (!FAST) coefs(sT[cl]);
                    const r4<R> qd = sQ[cl];
                    R fkl = 0, fkr = 0, fhl = 0, fhr = 0;
                    if (MODE == M_SI) {
                        load_phi4<R>(phr, cell, fkl, fkr, fhl, fhr);
                        fkl *= cs; fkr *= cs; fhl *= cs; fhr *= cs;
                    }
    #pragma unroll
                    for (int t = 0; t < PPL; ++t) {
                        const int pp = ls + LPC * t;
                        if (pp >= P) continue;
                        const Coef<R> &a = ac[t];
                        const r2<R> inP = (!FAST && refl_l && cell == 0)
                                              ? face_ld_M((size_t)pp)
                                              : (IN_BF ? unpack_bf16x2(hsP[cl * P + pp]) : sP[cl * P + pp]);
                        const r2<R> inM = (!FAST && refl_r && cell == J - 1)
                                              ? face_ld_P((size_t)J * P + pp)
                                              : (IN_BF ? unpack_bf16x2(hsM[cl * P + pp]) : sM[cl * P + pp]);
                        r4<R> *slot = const_cast<r4<R> *>(sE) + cl * P + pp;  // this lane's own (cell, pair) slot
                        const r4<R> pe = *slot;                               // psi_{k-1/2} (M_LIN: r0)
                        PairRhs<R> u = MODE == M_LIN ? PairRhs<R>{0, 0, 0, 0, 0, 0, 0, 0} : pair_rhs_fixed(qd, ce, pe);
                        r4<R> yo;
                        if (MODE == M_SI) {
                            // outgoing part of A^{-1} c_fixed; the next sweep's offset adds
                            // s (A^{-1} phi^{l+1})_out in phase E
                            yo.x = a.pr * u.uki + a.pi * u.ukr + a.rr * u.uhi + a.ri * u.uhr;
                            yo.y = a.ur * u.uki + a.ui * u.ukr + a.vr * u.uhi + a.vi * u.uhr;
                            yo.z = a.pr * u.vkr - a.pi * u.vki + a.rr * u.vhr - a.ri * u.vhi;
                            yo.w = a.ur * u.vkr - a.ui * u.vki + a.vr * u.vhr - a.vi * u.vhi;
                            u.ukr += fkl; u.uki += fkr; u.uhr += fhl; u.uhi += fhr;
                            u.vkr += fkl; u.vki -= fkr; u.vhr += fhl; u.vhi -= fhr;
                            if (!FAST && cell == J - 1 && p.bc_right == BC_REFLECT)
                                st2(p.refl + pp, ld2(fPr + (size_t)J * P + pp).x, ld2(fPr + (size_t)J * P + pp).y);
                        }
                        u.ukr += mw[t].x * inP.x; u.uhr += mw[t].x * inP.y;
                        u.vki -= mw[t].x * inM.x; u.vhi -= mw[t].x * inM.y;
                        R ykr, yki, yhr, yhi, zkr, zki, zhr, zhi;
                        ainv(a, u.ukr, u.uki, u.uhr, u.uhi, ykr, yki, yhr, yhi);
                        ainv(a, u.vkr, u.vki, u.vhr, u.vhi, zkr, zki, zhr, zhi);
                        if (MODE != M_SI) {  // outgoing corners of y (M_LIN: plus r0)
                            yo = r4<R>{yki, yhi, zkr, zhr};
                            if (MODE == M_LIN) { yo.x += pe.x; yo.y += pe.y; yo.z += pe.z; yo.w += pe.w; }
                        }
                        *slot = yo;  // phase E reads it back; no other lane touches this slot
                        m0 += mw[t].y * (ykr + zkr); m1 += mw[t].y * (yki - zki);
                        m2 += mw[t].y * (yhr + zhr); m3 += mw[t].y * (yhi - zhi);
                    }
                }
                *reinterpret_cast<float4 *>(xp + xpose_idx(lane, 4 * r)) = make_float4(m0, m1, m2, m3);
            }
            };
            if (fast) phase_a(BoolTag<true>{});
            else phase_a(BoolTag<false>{});
            __syncwarp();
            // ---------------- phase B: each lane sums the LPC lane partials of the
            // (segment, moment) values it owns, compensated (Kahan)
            ff own[NOWN];
    #pragma unroll
            for (int k = 0; k < NOWN; ++k) {
                const int f = lane * NOWN + k;
                const int g = f / V, v = f % V;  // segment and value index (row * 4 + moment)
                // KC interleaved Kahan sums over the segment's lanes, joined exactly
                constexpr int KC = LPC >= 4 ? 4 : LPC;
                float sk[KC], ck[KC];
    #pragma unroll
                for (int a = 0; a < KC; ++a) { sk[a] = 0.f; ck[a] = 0.f; }
                if (g < SPW) {
    #pragma unroll
                    for (int q = 0; q < LPC; q += KC) {
    #pragma unroll
                        for (int a = 0; a < KC; ++a) {
                            const float x = xp[xpose_idx(g * LPC + q + a, v)];
                            const float y = __fsub_rn(x, ck[a]);
                            const float t = __fadd_rn(sk[a], y);
                            ck[a] = __fsub_rn(__fsub_rn(t, sk[a]), y);
                            sk[a] = t;
                        }
                    }
                }
                ff acc = ff_norm(sk[0], -ck[0]);
    #pragma unroll
                for (int a = 1; a < KC; ++a) acc = ff_add(acc, ff_norm(sk[a], -ck[a]));
                own[k] = acc;
            }
            __syncwarp();
            // ---------------- phase C: capacitance solve + residual, in double
    #pragma unroll
            for (int k = 0; k < NOWN; ++k) {
                const int f = lane * NOWN + k;
                const int g = f / V, v = f % V;
                const int row = v >> 2, comp = v & 3;
                const int cell = chunk * CPC + row * SPW + g;
                ff phi;
                if (MODE != M_SI) {
                    ff r_par;
                    if constexpr (NOWN >= 4) {
                        r_par = own[k ^ 2];
                    } else {
                        constexpr int o = NOWN == 2 ? 1 : 2;
                        r_par.h = __shfl_xor_sync(FULL, own[k].h, o);
                        r_par.l = __shfl_xor_sync(FULL, own[k].l, o);
                    }
                    const int m = (g < SPW && cell < J) ? sT[row * SPW + g] : 0;
                    if (m != mK) {  // capacitance of this value's material (cached per lane)
                        mK = m;
                        kA = __ldg(p.matKf + 2 * m);
                        kB = __ldg(p.matKf + 2 * m + 1);
                    }
                    phi = comp < 2 ? ff_add(ff_mul(ff{kA.x, kA.y}, own[k]), ff_mul(ff{kA.z, kA.w}, r_par))
                                   : ff_add(ff_mul(ff{kB.x, kB.y}, r_par), ff_mul(ff{kB.z, kB.w}, own[k]));
                } else {
                    phi = own[k];
                }
                if (g < SPW && cell < J) {
                    const float2 old = old_phi[k];
                    const float d = ff_diff(phi, ff{old.x, old.y});
                    accf_d2 = __fmaf_rn(d, d, accf_d2);
                    // norm of the whole iterate (M_LIN: phi(h0) + correction)
                    const float tot = MODE == M_LIN ? __fadd_rn(ref_phi[k].x, phi.h) : phi.h;
                    accf_p2 = __fmaf_rn(tot, tot, accf_p2);
                    phw[4 * (size_t)cell + comp] = make_float2(phi.h, phi.l);
                    xp[g * V + v] = __fadd_rn(phi.h, phi.l);  // phi of (segment g, value v) for phase D
                }
            }
            __syncwarp();
            // ---------------- phase D/E: outgoing corners = y_out + s (A^{-1} Phi)_out
            auto phase_e = [&](auto fast_tag) {
            constexpr bool FAST = decltype(fast_tag)::value;
    #pragma unroll
            for (int r = 0; r < CHUNK; ++r) {
                const int cl = r * SPW + seg;
                const int cell = chunk * CPC + cl;
                if (!FAST && cell >= J) continue;
                if (!FAST) coefs(sT[cl]);
                const float4 F = *reinterpret_cast<const float4 *>(xp + seg * V + 4 * r);
                const R Fkl = F.x * cs, Fkr = F.y * cs, Fhl = F.z * cs, Fhr = F.w * cs;
    #pragma unroll
                for (int t = 0; t < PPL; ++t) {
                    const int pp = ls + LPC * t;
                    if (pp >= P) continue;
                    const Coef<R> &a = ac[t];
                    const r4<R> yo = sE[cl * P + pp];
                    // +mu: Im(A^{-1} s Phi); -mu: Re(A^{-1} s conj(Phi))
                    const R ok = yo.x + (a.pr * Fkr + a.pi * Fkl + a.rr * Fhr + a.ri * Fhl);
                    const R oh = yo.y + (a.ur * Fkr + a.ui * Fkl + a.vr * Fhr + a.vi * Fhl);
                    const R mk = yo.z + (a.pr * Fkl + a.pi * Fkr + a.rr * Fhl + a.ri * Fhr);
                    const R mh = yo.w + (a.ur * Fkl + a.ui * Fkr + a.vr * Fhl + a.vi * Fhr);
                    if (OUT_BF) {
                        hPw[(size_t)(cell + 1) * P + pp] = pack_bf16x2(ok, oh);
                        hMw[(size_t)cell * P + pp] = pack_bf16x2(mk, mh);
                    } else if (PING) {
                        st2(fPw + (size_t)(cell + 1) * P + pp, ok, oh);
                        st2(fMw + (size_t)cell * P + pp, mk, mh);
                    } else {
                        st4(p.g + (size_t)pp * J + cell, ok, oh, mk, mh);
                    }
                }
            }
            };
            if (fast) phase_e(BoolTag<true>{});
            else phase_e(BoolTag<false>{});
            fence_proxy_async();  // this lane's phase-A stores into the ring before the next copy into it
            __syncwarp();  // stage i and the transpose buffer fully read
            if constexpr (ASYNC) {
                if (!prev_known && i + 1 < nmine) {
                    int known = 0;  // 1: the previous iteration goes on, 2: it was the last
                    if (lane == 0 && poll_tag == (unsigned)rep) {
                        asm volatile("fence.acq_rel.gpu;\n" ::: "memory");
                        known = *(volatile const int *)&p.as->rec[(rep - 1) & 3].status == ST_RUNNING ? 1 : 2;
                    }
                    known = __shfl_sync(FULL, known, 0);
                    if (known == 1) prev_known = true;
                    if (known == 2) {
                        // drop the rest of this speculative iteration, once the
                        // copies already issued for the next chunks have landed
                        const int last = i + STAGES < nmine ? i + STAGES : nmine;
                        for (int k = i + 1; k < last; ++k) (void)mbar_wait(bars + stage_of(k), parity_of(k));
                        consumed = last;
                        if (lane == 0) s_stop[rep & 1] = 1;
                        break;
                    }
                }
            }
        }
        if (!ok_all) {
            // a copy never completed: record it and wait (bounded) for this warp's
            // outstanding copies before the block's shared memory is released
            if (lane == 0) atomicExch(&p.st->status, ST_TIMEOUT);
            // copies were issued for positions broke_at .. broke_at + STAGES - 1
            const int last = broke_at + STAGES - 1 < nmine ? broke_at + STAGES - 1 : nmine - 1;
            for (int k = broke_at; k <= last; ++k) (void)mbar_wait(bars + stage_of(k), parity_of(k));
        }
        if constexpr (!LOOP) {
            finalize_iteration((double)accf_d2, (double)accf_p2, p.partials, p.st, p.cfg, iter, p.use_cond, p.cond,
                               HALO == 1 ? 1 : (HALO == 3 ? 3 : (MODE == M_LIN ? 4 : 0)));
            return;
        } else if constexpr (ASYNC) {
            // the warp's partial, added up by the block at the top of the next
            // iteration; a copy that never completed stops the step
            rp += consumed;
            const double wd2 = warp_sum((double)accf_d2), wp2 = warp_sum((double)accf_p2);
            if (lane == 0) {
                s_wpart[rep & 1][warp][0] = wd2;
                s_wpart[rep & 1][warp][1] = wp2;
                s_wpart[rep & 1][warp][2] = ok_all ? 0.0 : 1.0;
                if (!ok_all) s_stop[rep & 1] = 1;
            }
            iter += 1;
        } else {
            rp += nmine;
            // per-warp partials and copy status, one block barrier; then thread 0
            // alone meets the grid
            __shared__ double s_wd[2][32];
            __shared__ int s_wok[32];
            __shared__ double s_ab[2];
            __shared__ int s_flag[2];  // grid barrier reached; some block reported a copy timeout
            const double wd2 = warp_sum((double)accf_d2), wp2 = warp_sum((double)accf_p2);
            if (lane == 0) {
                s_wd[0][warp] = wd2;
                s_wd[1][warp] = wp2;
                s_wok[warp] = ok_all ? 1 : 0;
            }
            __syncthreads();
            bool block_ok = true;
            for (int w = 0; w < wpb; ++w) block_ok = block_ok && s_wok[w] != 0;
            // the next iteration's invariant copies go out before the barrier
            if (lane == 0 && block_ok)
                for (int i = 0; i < STAGES - 1; ++i) issue_static(i);
            const int G = gridDim.x;
            double *lp = p.loop_partials + (size_t)(iter & 1) * 3 * G;
            const IterConfig *cfg = p.cfg;
            if (threadIdx.x == 0) {
                double d2 = 0.0, p2 = 0.0;
                for (int w = 0; w < wpb; ++w) {
                    d2 += s_wd[0][w];
                    p2 += s_wd[1][w];
                }
                lp[3 * blockIdx.x] = d2;
                lp[3 * blockIdx.x + 1] = p2;
                lp[3 * blockIdx.x + 2] = block_ok ? 0.0 : 1.0;
                s_flag[0] = grid_arrive_wait(p.loop_bar, (unsigned)(rep + 1) * (unsigned)G + (unsigned)cfg->bar_shortfall,
                                             cfg->bar_poll_limit ? cfg->bar_poll_limit : kWaitLimit) ? 1 : 0;
            }
            __syncthreads();
            const bool bar_ok = s_flag[0] != 0;
            // the next iteration's first incident faces go out now, their latency
            // hidden by the reduction and decision below (waited for if the step
            // ends here); the generic stores of the other blocks are ordered by
            // the grid barrier, the proxy fence orders them before the bulk reads
            if (lane == 0 && block_ok) {
                const int nfrd = PING ? ((base + iter + 1) & 1) : base;
                asm volatile("fence.proxy.async.global;\n" ::: "memory");
                for (int i = 0; i < STAGES - 1 && i < nmine; ++i) {
                    const int c0 = chunk_of(i) * CPC;
                    const int nv = J - c0 < CPC ? J - c0 : CPC;
                    unsigned char *stg = ring + (size_t)stage_of(i) * sbytes;
                    unsigned long long *bar = bars + stage_of(i);
                    const unsigned bF = round16(nv * P * FB);
                    const void *srcP = IN_BF ? (const void *)(p.hfP[nfrd] + (size_t)c0 * P)
                                             : (const void *)(p.faceP[nfrd] + (size_t)c0 * P);
                    const void *srcM = IN_BF ? (const void *)(p.hfM[nfrd] + (size_t)(c0 + 1) * P)
                                             : (const void *)(p.faceM[nfrd] + (size_t)(c0 + 1) * P);
                    mbar_expect_tx_arrive(bar, 2 * bF);
                    bulk_g2s(stg + oP, srcP, bF, bar);
                    bulk_g2s(stg + oM, srcM, bF, bar);
                }
            }
            // every block sums the partials in the same fixed order (warp 0)
            if (warp == 0) {
                double a = 0.0, b = 0.0, f = 0.0;
                for (int q = lane; q < G; q += 32) {
                    a += __ldcg(lp + 3 * q);
                    b += __ldcg(lp + 3 * q + 1);
                    f += __ldcg(lp + 3 * q + 2);
                }
                a = warp_sum(a);
                b = warp_sum(b);
                f = warp_sum(f);
                if (lane == 0) {
                    s_ab[0] = a;
                    s_ab[1] = b;
                    s_flag[1] = f != 0.0 ? 1 : 0;
                }
            }
            __syncthreads();
            const double a = s_ab[0], b = s_ab[1];
            const bool fault = s_flag[1] != 0 || !bar_ok;
            const int it = iter + 1;
            double resid;
            const int ns = loop_decision(a, b, fault, it, fixed_left, HALO == 2, cfg, stall, best, resid);
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                IterState *sw = p.st;
                sw->iter = it;
                sw->resid = resid;
                sw->d2 = a;
                sw->p2 = b;
                sw->stall = stall;
                sw->best = best;
                sw->launches += 1;
                if (ns != ST_TIMEOUT || sw->status == ST_RUNNING) sw->status = ns;
            }
            iter = it;
            status = ns;
            if (status != ST_RUNNING || it == cfg->pause_at) {
                // the next iteration's first copies (invariant part and faces) are
                // in flight: wait for them before the block's shared memory goes
                if (block_ok)
                    for (int i = 0; i < STAGES - 1 && i < nmine; ++i) (void)mbar_wait(bars + stage_of(i), parity_of(i));
                if constexpr (HALO == 0) {
                    // End of the step in the same launch (multiple balance: psi_{k+1/2}
                    // of every ordinate and corner, A^{-1}(c + s phi) with the incident
                    // faces the last iteration read, becomes psi_edge; its outgoing
                    // corners are the next step's initial iterate; phi is published).
                    // Every block took the same decision, and the faces the last
                    // iteration read (buffer frd_last) and its moments were complete at
                    // the grid barrier above.  Each warp streams its own chunks through
                    // its ring again, so the pass runs at the iteration's memory-level
                    // parallelism.  It writes psi_edge of its own cells and the other
                    // face buffer, which other blocks' discarded prefetches may still be
                    // reading.
                    if (p.loop_commit && status != ST_RUNNING) {
                        const bool go = status == ST_CONVERGED || (status == ST_MAXITER && cfg->commit_unconverged);
                        const int frd_l = (base + it - 1) & 1, fgs = frd_l ^ 1;
                        if (blockIdx.x == 0 && threadIdx.x == 0) {
                            p.st->committed = go ? 1 : 0;
                            p.st->base_next = go ? fgs : base;
                        }
                        if (go && block_ok) {
                            rp += STAGES - 1;  // the prefetched positions are spent; their data is not used
                            ring_commit(frd_l, fgs, p.phi[it & 1]);
                        }
                    }
                }
                return;
            }
        }
    }
    if constexpr (ASYNC) {
        // every warp has left the loop (with no copy in flight): one grid
        // barrier, then the end of the step over all cells
        __syncthreads();
        __shared__ int s_exit_ok;
        if (threadIdx.x == 0) {
            const bool ok = grid_arrive_wait(&p.as->exit_bar, (unsigned)gridDim.x + shortfall, wlimit);
            if (!ok) atomicExch(&p.st->status, ST_TIMEOUT);
            s_exit_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_exit_ok) return;
        IterState *st = p.st;
        const int fst = *(volatile const int *)&st->status, fit = *(volatile const int *)&st->iter;
        const bool go = fit >= 1 && (fst == ST_CONVERGED || (fst == ST_MAXITER && p.cfg->commit_unconverged));
        // the last iteration read buffer (base + fit - 1) % 3; the next step's
        // initial iterate goes to one of buffers 0 and 1 other than that one
        const int frd_last = (base + fit - 1) % 3;
        const int g_buf = frd_last == 2 ? 0 : 1 - frd_last;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->committed = go ? 1 : 0;
            st->base_next = go ? g_buf : base;
            st->rot3 = 1;
            st->cur_face = (base + fit) % 3;
        }
        if (!go) return;
        ring_commit(frd_last, g_buf, p.phi[fit & 1]);
    }
}

// ---------------------------------------------------------------------------
// Per-cell passes without reductions (LPC lanes per cell, PPL pairs per lane):
//   C_COMMIT_OCI / C_COMMIT_SI: if the step is accepted, the end-of-step flux
//     psi_{k+1/2} of every ordinate and corner, psi = A^{-1}(c + s phi), goes to
//     psi_edge (multiple balance: it is the next step's psi_{k-1/2}); the next
//     step's initial iterate (both time moments = psi_{k+1/2} at the faces)
//     goes to the free face buffer; phi is published.
//   C_SI_PREP: affine offsets g of the first sweep of a step from phi^(0).
//   C_GUESS : initial iterate from psi_edge (after set_state or a rejected step).
// ---------------------------------------------------------------------------
template <typename R, int LPC, int PPL, int MODE>
__device__ __forceinline__ void percell_body(const KParams<R> &p, int gw, int nwarps, int frd, int fgs,
                                             const phi_t<R> *phi_psi, const phi_t<R> *phi_pub);

template <typename R, int LPC, int PPL, int MODE>
__global__ void __launch_bounds__(256) k_percell(const KParams<R> p)
{
    IterState *st = p.st;
    const int status = st->status, iter = st->iter, base = st->base;
    bool go = true;
    int frd = 0, fgs = 0;
    const phi_t<R> *phi_psi = nullptr, *phi_pub = nullptr;
    constexpr bool COMMIT = MODE == C_COMMIT_OCI || MODE == C_COMMIT_SI || MODE == C_COMMIT_LIN;
    if (COMMIT) {
        go = iter >= 1 && (status == ST_CONVERGED || (status == ST_MAXITER && p.cfg->commit_unconverged));
        if (MODE == C_COMMIT_OCI || MODE == C_COMMIT_LIN) {
            frd = (base + iter - 1) & 1;
            fgs = frd ^ 1;
            phi_psi = p.phi[iter & 1];
        } else {
            frd = base;
            fgs = base ^ 1;
            phi_psi = (iter - 1 == 0) ? p.phi0 : p.phi[(iter - 1) & 1];
        }
        phi_pub = p.phi[iter & 1];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->committed = go ? 1 : 0;
            st->base_next = go ? fgs : base;
        }
    } else if (MODE == C_SI_PREP) {
        frd = base;
        phi_psi = p.phi0;
    } else {  // C_GUESS
        fgs = st->base_next;
    }
    if (!go) return;
    percell_body<R, LPC, PPL, MODE>(p, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, (gridDim.x * blockDim.x) >> 5,
                                    frd, fgs, phi_psi, phi_pub);
}

// The per-cell work of k_percell for warp gw of nwarps, face buffers frd (read)
// and fgs (written); also the end of a step of the barrier-free loop, so every
// load of data written during the launch goes through L2 (ld.cg).
template <typename R, int LPC, int PPL, int MODE>
__device__ __forceinline__ void percell_body(const KParams<R> &p, int gw, int nwarps, int frd, int fgs,
                                             const phi_t<R> *phi_psi, const phi_t<R> *phi_pub)
{
    constexpr int SPW = 32 / LPC;
    constexpr int ROWS = 4;  // cells per segment in flight per pass (loads issued together)
    constexpr bool COMMIT = MODE == C_COMMIT_OCI || MODE == C_COMMIT_SI || MODE == C_COMMIT_LIN;
    const int lane = threadIdx.x & 31;
    const int seg = lane / LPC, ls = lane % LPC;
    const int J = p.J, P = p.P;
    const bool refl_l = (MODE == C_COMMIT_OCI || MODE == C_COMMIT_LIN) && p.bc_left == BC_REFLECT;
    const bool refl_r = (MODE == C_COMMIT_OCI || MODE == C_COMMIT_LIN) && p.bc_right == BC_REFLECT;
    const bool ext = (MODE == C_COMMIT_OCI || MODE == C_COMMIT_SI || MODE == C_COMMIT_LIN) && p.cfg->extrap != 0;
    R mu[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) mu[i] = (ls + LPC * i < P) ? ldg2(p.muw + ls + LPC * i).x : R(0);
    // a pass covers ROWS rows of SPW cells per warp
    for (int c0 = gw * SPW * ROWS; c0 < J; c0 += nwarps * SPW * ROWS) {
        int cellr[ROWS], mr[ROWS];
        r4<R> qdr[ROWS];
        R F[ROWS][4];
        r4<R> per[ROWS][PPL];
        r2<R> inPr[ROWS][PPL], inMr[ROWS][PPL];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int cell = c0 + r * SPW + seg;
            cellr[r] = cell;
            const bool valid = cell < J;
            mr[r] = valid ? __ldg(p.mat + cell) : 0;
            qdr[r] = valid ? ldg4(p.cellq + cell) : r4<R>{0, 0, 0, 0};
            F[r][0] = F[r][1] = F[r][2] = F[r][3] = 0;
            if (MODE != C_GUESS && valid) load_phi4<R>(phi_psi, cell, F[r][0], F[r][1], F[r][2], F[r][3]);
            if (MODE == C_COMMIT_LIN && valid) {
                R a0, a1, a2, a3;
                load_phi4<R>(reinterpret_cast<const phi_t<R> *>(p.phi_ref), cell, a0, a1, a2, a3);
                F[r][0] += a0; F[r][1] += a1; F[r][2] += a2; F[r][3] += a3;
            }
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                const int pp = ls + LPC * i;
                const bool ok = valid && pp < P;
                per[r][i] = ok ? ldcg4(p.psi_edge + (size_t)cell * P + pp) : r4<R>{0, 0, 0, 0};
                inPr[r][i] = inMr[r][i] = r2<R>{0, 0};
                if (ok && COMMIT) {
                    inPr[r][i] = (refl_l && cell == 0) ? ldcg2(p.faceM[frd] + pp) : ldcg2(p.faceP[frd] + (size_t)cell * P + pp);
                    inMr[r][i] = (refl_r && cell == J - 1) ? ldcg2(p.faceP[frd] + (size_t)J * P + pp)
                                                          : ldcg2(p.faceM[frd] + (size_t)(cell + 1) * P + pp);
                    if (MODE == C_COMMIT_LIN) {  // incident h0 + d
                        const r2<R> a = (refl_l && cell == 0) ? ldcg2(p.h0M + pp) : ldcg2(p.h0P + (size_t)cell * P + pp);
                        const r2<R> b = (refl_r && cell == J - 1) ? ldcg2(p.h0P + (size_t)J * P + pp)
                                                                 : ldcg2(p.h0M + (size_t)(cell + 1) * P + pp);
                        inPr[r][i].x += a.x; inPr[r][i].y += a.y;
                        inMr[r][i].x += b.x; inMr[r][i].y += b.y;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int cell = cellr[r];
            if (cell >= J) continue;
            const int m = mr[r];
            const r4<R> qd = qdr[r];
            const r2<R> es = ldg2(p.matpar + m);
            const R Fkl = F[r][0] * es.y, Fkr = F[r][1] * es.y, Fhl = F[r][2] * es.y, Fhr = F[r][3] * es.y;
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                const int pp = ls + LPC * i;
                if (pp >= P) continue;
                const r4<R> pe = per[r][i];
                if (MODE == C_GUESS) {
                    st2(p.faceP[fgs] + (size_t)(cell + 1) * P + pp, pe.y, pe.y);
                    st2(p.faceM[fgs] + (size_t)cell * P + pp, pe.z, pe.z);
                    continue;
                }
                const Coef<R> a = load_coef(p.tab, m, P, pp);
                R ukr = qd.x + es.x * pe.x + Fkl, uki = qd.y + es.x * pe.y + Fkr, uhr = qd.z + Fhl, uhi = qd.w + Fhr;
                R vkr = qd.x + es.x * pe.z + Fkl, vki = -(qd.y + es.x * pe.w) - Fkr, vhr = qd.z + Fhl, vhi = -qd.w - Fhr;
                if (MODE == C_SI_PREP) {
                    const R ok = a.pr * uki + a.pi * ukr + a.rr * uhi + a.ri * uhr;
                    const R oh = a.ur * uki + a.ui * ukr + a.vr * uhi + a.vi * uhr;
                    const R mk = a.pr * vkr - a.pi * vki + a.rr * vhr - a.ri * vhi;
                    const R mh = a.ur * vkr - a.ui * vki + a.vr * vhr - a.vi * vhi;
                    st4(p.g + (size_t)pp * J + cell, ok, oh, mk, mh);
                    if (cell == J - 1 && p.bc_right == BC_REFLECT) {
                        // SI lags a reflecting right face: the first sweep sees the
                        // initial iterate's outgoing +mu flux there.
                        const r2<R> v = ldcg2(p.faceP[frd] + (size_t)J * P + pp);
                        st2(p.refl + pp, v.x, v.y);
                    }
                    continue;
                }
                // end-of-step components only (k+1/2): second rows of A^{-1}
                R phr_, phi_, mhr, mhi;
                commit_corners<R>(a, qd, es.x, pe, Fkl, Fkr, Fhl, Fhr, mu[i], inPr[r][i], inMr[r][i], phr_, phi_, mhr,
                                  mhi);
                // psi+ = (L, R) = (Re, Im); psi- = conj(z): (Re z, -Im z)
                st4(p.psi_edge + (size_t)cell * P + pp, phr_, phi_, mhr, -mhi);
                if (ext) {  // linear in time through the previous end-of-step flux pe
                    const R dP = phi_ - pe.y, dM = mhr - pe.z;
                    st2(p.faceP[fgs] + (size_t)(cell + 1) * P + pp, phi_ + R(0.5) * dP, phi_ + dP);
                    st2(p.faceM[fgs] + (size_t)cell * P + pp, mhr + R(0.5) * dM, mhr + dM);
                } else {
                    st2(p.faceP[fgs] + (size_t)(cell + 1) * P + pp, phi_, phi_);
                    st2(p.faceM[fgs] + (size_t)cell * P + pp, mhr, mhr);
                }
            }
            if (MODE == C_COMMIT_SI && ext) {
                // an SI step starts from its scalar flux: extrapolate it in time as the faces
                double old2, old3;
                prev_end_moments(p.phi_out + 4 * (size_t)cell,
                                 LPC == 32 ? 0xffffffffu : (((1u << LPC) - 1u) << (seg * LPC)), seg * LPC, ls, old2, old3);
                for (int c = ls; c < 4; c += LPC) {
                    p.phi_out[4 * (size_t)cell + c] = PhiStore<R>::wide(__ldcg(phi_pub + 4 * (size_t)cell + c));
                    const double nh = PhiStore<R>::wide(__ldcg(phi_pub + 4 * (size_t)cell + 2 + (c & 1)));
                    const double old = (c & 1) ? old3 : old2;
                    p.phi0[4 * (size_t)cell + c] = phi_from_double<R>(nh + (c < 2 ? 0.5 : 1.0) * (nh - old));
                }
            } else if (MODE == C_COMMIT_OCI || MODE == C_COMMIT_SI) {
                for (int c = ls; c < 4; c += LPC) {
                    p.phi_out[4 * (size_t)cell + c] = PhiStore<R>::wide(__ldcg(phi_pub + 4 * (size_t)cell + c));
                    p.phi0[4 * (size_t)cell + c] = __ldcg(phi_pub + 4 * (size_t)cell + 2 + (c & 1));
                }
            }
            if constexpr (MODE == C_COMMIT_LIN && sizeof(R) == 4) {
                for (int c = ls; c < 4; c += LPC) {
                    const float2 a = __ldcg(phi_pub + 4 * (size_t)cell + c), b = p.phi_ref[4 * (size_t)cell + c];
                    p.phi_out[4 * (size_t)cell + c] = (double)a.x + (double)a.y + (double)b.x + (double)b.y;
                    const float2 ah = __ldcg(phi_pub + 4 * (size_t)cell + 2 + (c & 1));
                    const float2 bh = p.phi_ref[4 * (size_t)cell + 2 + (c & 1)];
                    const ff t = ff_add(ff{ah.x, ah.y}, ff{bh.x, bh.y});
                    p.phi0[4 * (size_t)cell + c] = make_float2(t.h, t.l);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Learned-guess lift: move an iterate toward a predicted scalar flux phat by
// adding the isotropic correction (phat - phi)/2 of each upstream corner to
// every incident angular flux it feeds (an isotropic angular flux psi = phi/2
// carries scalar flux phi with weights summing to 2), and make phat the
// iterate's scalar flux.  LIFT_GUESS works on the step's initial iterate
// (faces[base_next], phi0); LIFT_CORR on the current iterate of a paused step
// (faces[(base + iter) & 1], phi[iter & 1]).  One warp row per cell.
// ---------------------------------------------------------------------------
enum : int { LIFT_GUESS = 0, LIFT_CORR = 1 };

template <typename R, int LPC, int PPL, int MODE>
__global__ void __launch_bounds__(256) k_lift(const KParams<R> p, const double *__restrict__ phat,
                                              const double *__restrict__ hist0, const double *__restrict__ hist1)
{
    constexpr int SPW = 32 / LPC;
    const int lane = threadIdx.x & 31;
    const int seg = lane / LPC, ls = lane % LPC;
    const int J = p.J, P = p.P;
    const IterState *st = p.st;
    int fb;
    phi_t<R> *ph;
    if (MODE == LIFT_GUESS) {
        fb = st->base_next;
        ph = p.phi0;
    } else {
        fb = (st->base + st->iter) & 1;
        ph = p.phi[st->iter & 1];
    }
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int cell = gw * SPW + seg; cell - seg < J; cell += nwarps * SPW) {
        const bool valid = cell < J;  // all lanes stay in the loop body (warp barriers below)
        double d[4] = {0.0, 0.0, 0.0, 0.0};
        if (valid) {
            // the iterate's moments: phi0, or with the initial iterate extrapolated in
            // time, the same extrapolation of the last two committed end-of-step moments
            const bool ext = MODE == LIFT_GUESS && p.cfg->extrap != 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                double it;
                if (ext) {
                    const double e1 = hist0[4 * (size_t)cell + 2 + (c & 1)], e2 = hist1[4 * (size_t)cell + 2 + (c & 1)];
                    it = e1 + (c < 2 ? 0.5 : 1.0) * (e1 - e2);
                } else {
                    it = PhiStore<R>::wide(ph[4 * (size_t)cell + c]);
                }
                d[c] = phat[4 * (size_t)cell + c] - it;
            }
        }
        __syncwarp();
        if (!valid) continue;
#pragma unroll
        for (int i = 0; i < PPL; ++i) {
            const int pp = ls + LPC * i;
            if (pp >= P) continue;
            r2<R> *fp = p.faceP[fb] + (size_t)(cell + 1) * P + pp;  // +mu leaves through the right face (corner R)
            r2<R> *fm = p.faceM[fb] + (size_t)cell * P + pp;        // -mu leaves through the left face (corner L)
            const r2<R> a = *fp, b = *fm;
            *fp = r2<R>{a.x + (R)(0.5 * d[1]), a.y + (R)(0.5 * d[3])};
            *fm = r2<R>{b.x + (R)(0.5 * d[0]), b.y + (R)(0.5 * d[2])};
        }
        // the lanes of a cell belong to one segment: after their reads above,
        // its first lanes overwrite the cell's moments
        for (int c = ls; c < 4; c += LPC) ph[4 * (size_t)cell + c] = phi_from_double<R>(phat[4 * (size_t)cell + c]);
    }
}

// ---------------------------------------------------------------------------
// FP32 refinement, residual pass: one OCI application G(h0) evaluated in FP64
// from the saved FP32 halo h0 (same inputs the FP32 iteration uses), giving
// the high-precision residual r0 = G(h0) - h0 of every outgoing corner and the
// scalar flux phi(h0).  The correction d then solves d = B d + r0 in FP32,
// where B is the same OCI map with no source and homogeneous boundary data.
// ---------------------------------------------------------------------------
struct RefineArgs {
    const double *tab64;     // [n_mat][P][8] complex entries of A_{+mu}^{-1}
    const double *matpar64;  // [n_mat][2] (e, s)
    const double *muw64;     // [P][2]
    r4<float> *r0;           // out [J][P]
    float2 *phi_ref;         // out [J][4] double-float
};

template <int LPC, int PPL>
__global__ void __launch_bounds__(256) k_refine_residual(const KParams<float> p, const RefineArgs q)
{
    constexpr int SPW = 32 / LPC;
    const int lane = threadIdx.x & 31;
    const int seg = lane / LPC, ls = lane % LPC;
    const int J = p.J, P = p.P;
    const bool refl_l = p.bc_left == BC_REFLECT, refl_r = p.bc_right == BC_REFLECT;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c0 = gw * SPW; c0 < J; c0 += nwarps * SPW) {
        const int cell = c0 + seg;
        const bool valid = cell < J;
        const int m = valid ? __ldg(p.mat + cell) : 0;
        const double e = q.matpar64[2 * m], sc = q.matpar64[2 * m + 1];
        double qd[4] = {0, 0, 0, 0};
        if (valid) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(p.cellq + cell));
            qd[0] = v.x; qd[1] = v.y; qd[2] = v.z; qd[3] = v.w;
        }
        double u[PPL][8];
        double mom[4] = {0, 0, 0, 0};
#pragma unroll
        for (int t = 0; t < PPL; ++t) {
            const int pp = ls + LPC * t;
#pragma unroll
            for (int z = 0; z < 8; ++z) u[t][z] = 0.0;
            if (!(valid && pp < P)) continue;
            const double *a = q.tab64 + ((size_t)m * P + pp) * 8;
            const double mu = q.muw64[2 * pp], w = q.muw64[2 * pp + 1];
            const r2<float> inP = (refl_l && cell == 0) ? p.h0M[pp] : p.h0P[(size_t)cell * P + pp];
            const r2<float> inM = (refl_r && cell == J - 1) ? p.h0P[(size_t)J * P + pp] : p.h0M[(size_t)(cell + 1) * P + pp];
            const float4 pe = *reinterpret_cast<const float4 *>(p.psi_edge + (size_t)cell * P + pp);
            double *uu = u[t];
            uu[0] = qd[0] + e * pe.x + mu * inP.x; uu[1] = qd[1] + e * pe.y; uu[2] = qd[2] + mu * inP.y; uu[3] = qd[3];
            uu[4] = qd[0] + e * pe.z; uu[5] = -(qd[1] + e * pe.w + mu * inM.x); uu[6] = qd[2]; uu[7] = -(qd[3] + mu * inM.y);
            const Coef<double> c{a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7]};
            double ykr, yki, yhr, yhi, zkr, zki, zhr, zhi;
            ainv(c, uu[0], uu[1], uu[2], uu[3], ykr, yki, yhr, yhi);
            ainv(c, uu[4], uu[5], uu[6], uu[7], zkr, zki, zhr, zhi);
            mom[0] += w * (ykr + zkr); mom[1] += w * (yki - zki); mom[2] += w * (yhr + zhr); mom[3] += w * (yhi - zhi);
        }
#pragma unroll
        for (int o = LPC / 2; o >= 1; o >>= 1)
#pragma unroll
            for (int z = 0; z < 4; ++z) mom[z] += __shfl_xor_sync(FULL, mom[z], o);
        const kmat K = p.matK[m];
        const double phi[4] = {K.k00 * mom[0] + K.k01 * mom[2], K.k00 * mom[1] + K.k01 * mom[3],
                               K.k10 * mom[0] + K.k11 * mom[2], K.k10 * mom[1] + K.k11 * mom[3]};
        if (!valid) continue;
        const double Fkl = sc * phi[0], Fkr = sc * phi[1], Fhl = sc * phi[2], Fhr = sc * phi[3];
#pragma unroll
        for (int t = 0; t < PPL; ++t) {
            const int pp = ls + LPC * t;
            if (pp >= P) continue;
            const double *a = q.tab64 + ((size_t)m * P + pp) * 8;
            const double *uu = u[t];
            const double uk_i = uu[1] + Fkr, uk_r = uu[0] + Fkl, uh_i = uu[3] + Fhr, uh_r = uu[2] + Fhl;
            const double vk_r = uu[4] + Fkl, vk_i = uu[5] - Fkr, vh_r = uu[6] + Fhl, vh_i = uu[7] - Fhr;
            const double ok = a[0] * uk_i + a[1] * uk_r + a[2] * uh_i + a[3] * uh_r;
            const double oh = a[4] * uk_i + a[5] * uk_r + a[6] * uh_i + a[7] * uh_r;
            const double mk = a[0] * vk_r - a[1] * vk_i + a[2] * vh_r - a[3] * vh_i;
            const double mh = a[4] * vk_r - a[5] * vk_i + a[6] * vh_r - a[7] * vh_i;
            const r2<float> hp = p.h0P[(size_t)(cell + 1) * P + pp], hm = p.h0M[(size_t)cell * P + pp];
            q.r0[(size_t)cell * P + pp] = r4<float>{(float)(ok - hp.x), (float)(oh - hp.y), (float)(mk - hm.x), (float)(mh - hm.y)};
        }
        for (int cc = ls; cc < 4; cc += LPC) {
            const float h = (float)phi[cc];
            q.phi_ref[4 * (size_t)cell + cc] = make_float2(h, (float)(phi[cc] - (double)h));
        }
    }
}

// Step prologue: reset the iteration state for a new time step.
static __global__ void k_step_begin(IterState *st)
{
    if (st->chain) {  // queued behind the previous step: run only if that one committed cleanly
        st->chain = 0;
        if (!st->committed || st->status == ST_STALL) {
            st->status = ST_HELD;
            return;
        }
    }
    st->iter = 0;
    st->status = ST_RUNNING;
    st->arrive = 0u;
    st->launches = 0;
    st->base = st->base_next;
    st->resid = 0.0;
    st->stall = 0;
    st->best = __longlong_as_double(0x7ff0000000000000LL);
    st->rot3 = 0;
    st->cur_face = st->base;
    st->lin_first = 0;
}

// Resume a stalled step with the correction iteration: the high-precision
// residual pass counts as one iteration.
static __global__ void k_refine_setup(IterState *st)
{
    st->iter += 1;
    st->lin_first = st->iter + 1;
    st->status = ST_RUNNING;
    st->stall = 0;
    st->best = __longlong_as_double(0x7ff0000000000000LL);
    st->arrive = 0u;
}

// ---------------------------------------------------------------------------
// SI transport sweep (Sec. "Source Iteration"): for one ordinate, march the
// cells in the direction of travel.  With the lagged scattering source folded
// into g, the outgoing corner pair of cell j is an affine map of the incident
// pair: out = G in + g, G = mu [[Im P, Im Rr], [Im U, Im V]] (the same for
// +mu and -mu).  One warp per (pair, direction): the pair's G for every
// material sits in shared memory, the per-cell material ids and offsets g
// stream through a SI_NB-batch cp.async ring (32 cells per batch, one cell per
// lane), and lane 0 carries the dependent chain.  A reflecting left face needs
// the -mu sweep first, so then one warp runs both directions.
// ---------------------------------------------------------------------------
constexpr int SI_NB = 16;                 // ring depth in 32-cell batches
constexpr int SI_SMAT_BYTES = 32768;      // shared-memory table budget

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename R>
__device__ __forceinline__ void cp_async_r2(r2<R> *smem, const r2<R> *gmem)
{
    if constexpr (sizeof(R) == 4) cp_async8(smem, gmem);
    else cp_async16(smem, gmem);
}

template <typename R>
struct SiShared {
    static constexpr int SMAT = SI_SMAT_BYTES / (int)sizeof(r4<R>);
    r4<R> G[SMAT];                 // per material: mu (Im P, Im Rr, Im U, Im V)
    int mat[SI_NB][32];
    r2<R> g[SI_NB][32];
    r4<R> Gc[32];                  // G of the current batch's cells
    r2<R> out[32];
};

template <typename R>
__device__ __forceinline__ r4<R> si_G(const KParams<R> &p, const SiShared<R> &sh, int m, int pp, bool in_smem)
{
    if (in_smem) return sh.G[m];
    const Coef<R> a = load_coef(p.tab, m, p.P, pp);
    const R mu = ldg2(p.muw + pp).x;
    return r4<R>{mu * a.pi, mu * a.ri, mu * a.ui, mu * a.vi};
}

template <typename R>
__device__ void si_sweep(const KParams<R> &p, SiShared<R> &sh, int pp, int dir, int fb, R ink, R inh, bool in_smem)
{
    const int lane = threadIdx.x & 31;
    const int J = p.J, P = p.P;
    const int nb = (J + 31) / 32;
    // cell visited at sweep position t
    auto cell_at = [&](int t) { return dir > 0 ? t : J - 1 - t; };
    auto issue = [&](int b) {
        const int t = 32 * b + lane;
        if (b < nb && t < J) {
            const int j = cell_at(t);
            const int slot = b % SI_NB;
            cp_async4(&sh.mat[slot][lane], p.mat + j);
            const r2<R> *src = reinterpret_cast<const r2<R> *>(p.g + (size_t)pp * J + j) + (dir > 0 ? 0 : 1);
            cp_async_r2(&sh.g[slot][lane], src);
        }
        cp_async_commit();
    };
#pragma unroll 1
    for (int b = 0; b < SI_NB - 1; ++b) issue(b);
#pragma unroll 1
    for (int b = 0; b < nb; ++b) {
        issue(b + SI_NB - 1);
        cp_async_wait<SI_NB - 1>();
        __syncwarp();
        const int slot = b % SI_NB;
        const int n = J - 32 * b < 32 ? J - 32 * b : 32;
        if (lane < n) sh.Gc[lane] = si_G(p, sh, sh.mat[slot][lane], pp, in_smem);
        __syncwarp();
        if (lane == 0) {
            const r4<R> *Gc = sh.Gc;
            const r2<R> *gs = sh.g[slot];
            r2<R> *o = sh.out;
            // groups of 8 cells: all operands of a group are read before its
            // dependent chain runs and before its results are stored
#pragma unroll 1
            for (int k0 = 0; k0 < n; k0 += 8) {
                r4<R> G[8];
                r2<R> g[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = k0 + u < n ? k0 + u : n - 1;
                    G[u] = Gc[k];
                    g[u] = gs[k];
                }
                R ok[8], oh[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    ok[u] = G[u].x * ink + (G[u].y * inh + g[u].x);
                    oh[u] = G[u].z * ink + (G[u].w * inh + g[u].y);
                    if (k0 + u < n) { ink = ok[u]; inh = oh[u]; }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (k0 + u < n) o[k0 + u] = r2<R>{ok[u], oh[u]};
            }
        }
        __syncwarp();
        if (lane < n) {
            const int j = cell_at(32 * b + lane);
            const r2<R> o = sh.out[lane];
            if (dir > 0) st2(p.faceP[fb] + (size_t)(j + 1) * P + pp, o.x, o.y);
            else st2(p.faceM[fb] + (size_t)j * P + pp, o.x, o.y);
        }
        __syncwarp();
    }
    cp_async_wait<0>();
    __syncwarp();
}

template <typename R>
__global__ void __launch_bounds__(32) k_si_march(const KParams<R> p, int n_mat)
{
    __shared__ SiShared<R> sh;
    IterState *st = p.st;
    if (*(volatile int *)&st->status != ST_RUNNING) return;
    const int fb = *(volatile int *)&st->base;
    const int J = p.J, P = p.P;
    const int lane = threadIdx.x & 31;
    const bool both = p.bc_left == BC_REFLECT;
    const int pp = blockIdx.x % P;
    const int dir = both ? -1 : (blockIdx.x < P ? -1 : 1);
    const bool in_smem = n_mat <= SiShared<R>::SMAT;
    if (in_smem) {
        const R mu = ldg2(p.muw + pp).x;
        for (int m = lane; m < n_mat; m += 32) {
            const Coef<R> a = load_coef(p.tab, m, P, pp);
            sh.G[m] = r4<R>{mu * a.pi, mu * a.ri, mu * a.ui, mu * a.vi};
        }
    }
    __syncwarp();
    if (dir < 0) {
        // right face: prescribed / vacuum data, or (reflecting) the mirror
        // flux of the previous iterate, staged in refl by the previous pass;
        // it is copied into the face slot so later passes read what was used
        r2<R> in;
        if (p.bc_right == BC_REFLECT) {
            in = ld2(p.refl + pp);
            if (lane == 0) st2(p.faceM[fb] + (size_t)J * P + pp, in.x, in.y);
        } else {
            in = ld2(p.faceM[fb] + (size_t)J * P + pp);
        }
        si_sweep(p, sh, pp, -1, fb, in.x, in.y, in_smem);
    }
    if (both) {
        __syncwarp();
        const r2<R> v = ld2(p.faceM[fb] + pp);  // this sweep's -mu flux leaving through x = 0
        __syncwarp();
        if (lane == 0) st2(p.faceP[fb] + pp, v.x, v.y);
        si_sweep(p, sh, pp, 1, fb, v.x, v.y, in_smem);
    } else if (dir > 0) {
        const r2<R> in = ld2(p.faceP[fb] + pp);
        si_sweep(p, sh, pp, 1, fb, in.x, in.y, in_smem);
    }
}

// ---------------------------------------------------------------------------
// SI sweep as a parallel prefix over cells (an alternative to the sequential
// march above; the paper sweeps each ordinate cell by cell).  Along one
// ordinate's direction of travel the outgoing corner pair of cell j is an
// affine function of the pair entering it: x_j = G_j x_{j-1} + g_j, G_j the
// 2x2 response of the material (same as the march), g_j the offset the SI cell
// kernel stored.  Composition of affine maps is associative, so the chain of J
// cells is a scan: (1) every block composes a 2048-cell segment (256 threads x
// 8 cells, then a block scan of the thread maps) into one map per segment;
// (2) one warp per pair runs the segment maps from the boundary value (mu < 0
// first, so a reflecting left face takes this sweep's mu < 0 flux) and keeps
// each segment's entering value; (3) every block recomposes its segment and
// writes every cell's outgoing pair.  Chain ch = 2 pair + (0: mu < 0, 1: mu > 0).
// The association order differs from the march, so results agree with it to
// rounding, not bit for bit.
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 256, SCAN_CPT = 8, SCAN_SEG = SCAN_T * SCAN_CPT;

template <typename R>
struct Aff { R a, b, c, d, e, f; };  // x -> [[a, b], [c, d]] x + (e, f)

template <typename R>
__device__ __forceinline__ Aff<R> aff_id() { return {1, 0, 0, 1, 0, 0}; }

// the map "first, then second"
template <typename R>
__device__ __forceinline__ Aff<R> aff_then(const Aff<R> &f, const Aff<R> &s)
{
    return {s.a * f.a + s.b * f.c, s.a * f.b + s.b * f.d, s.c * f.a + s.d * f.c, s.c * f.b + s.d * f.d,
            s.a * f.e + (s.b * f.f + s.e), s.c * f.e + (s.d * f.f + s.f)};
}

template <typename R>
__device__ __forceinline__ Aff<R> aff_shfl_up(const Aff<R> &x, int d)
{
    return {__shfl_up_sync(FULL, x.a, d), __shfl_up_sync(FULL, x.b, d), __shfl_up_sync(FULL, x.c, d),
            __shfl_up_sync(FULL, x.d, d), __shfl_up_sync(FULL, x.e, d), __shfl_up_sync(FULL, x.f, d)};
}

template <typename R>
struct ScanShared {
    r2<R> g[SCAN_SEG];
    int mat[SCAN_SEG];
    Aff<R> warp_tot[SCAN_T / 32];
    Aff<R> block_tot;
};

// Stage the segment's offsets and materials, compose each thread's 8 cells
// and scan the thread maps over the block.  Returns the thread's exclusive
// prefix (maps of all earlier cells of the segment) and sets *total (block).
template <typename R>
__device__ Aff<R> scan_segment(const KParams<R> &p, ScanShared<R> &sh, int ch, int seg, Aff<R> *total)
{
    const int J = p.J, P = p.P;
    const int pp = ch >> 1, dir = (ch & 1) ? 1 : -1;
    const int s0 = seg * SCAN_SEG;
    const int n = J - s0 < SCAN_SEG ? J - s0 : SCAN_SEG;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int k = t; k < n; k += SCAN_T) {
        const int j = dir > 0 ? s0 + k : J - 1 - (s0 + k);
        sh.g[k] = reinterpret_cast<const r2<R> *>(p.g + (size_t)pp * J + j)[dir > 0 ? 0 : 1];
        sh.mat[k] = p.mat[j];
    }
    __syncthreads();
    const R mu = ldg2(p.muw + pp).x;
    int mc = -1;
    r4<R> G{0, 0, 0, 0};
    Aff<R> A = aff_id<R>();
    for (int i = 0; i < SCAN_CPT; ++i) {
        const int k = t * SCAN_CPT + i;
        if (k >= n) break;
        const int m = sh.mat[k];
        if (m != mc) {
            mc = m;
            const Coef<R> c = load_coef(p.tab, m, P, pp);
            G = r4<R>{mu * c.pi, mu * c.ri, mu * c.ui, mu * c.vi};
        }
        A = aff_then(A, Aff<R>{G.x, G.y, G.z, G.w, sh.g[k].x, sh.g[k].y});
    }
    // inclusive scan within the warp (earlier lanes' maps apply first)
    Aff<R> I = A;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const Aff<R> e = aff_shfl_up(I, d);
        if (lane >= d) I = aff_then(e, I);
    }
    if (lane == 31) sh.warp_tot[warp] = I;
    __syncthreads();
    // warp 0 scans the warp totals; slot w then holds the maps of warps 0..w-1
    constexpr int NW = SCAN_T / 32;
    if (warp == 0) {
        Aff<R> T = lane < NW ? sh.warp_tot[lane] : aff_id<R>();
#pragma unroll
        for (int d = 1; d < NW; d <<= 1) {
            const Aff<R> e = aff_shfl_up(T, d);
            if (lane >= d) T = aff_then(e, T);
        }
        Aff<R> X = aff_shfl_up(T, 1);
        if (lane == 0) X = aff_id<R>();
        __syncwarp();
        if (lane < NW) sh.warp_tot[lane] = X;
        if (lane == NW - 1) sh.block_tot = T;
    }
    __syncthreads();
    const Aff<R> W = sh.warp_tot[warp];  // maps of the earlier warps
    Aff<R> E = aff_shfl_up(I, 1);  // exclusive within the warp
    if (lane == 0) E = aff_id<R>();
    if (total) *total = sh.block_tot;
    return aff_then(W, E);
}

template <typename R>
__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const KParams<R> p, Aff<R> *__restrict__ agg)
{
    __shared__ ScanShared<R> sh;
    if (*(volatile int *)&p.st->status != ST_RUNNING) return;
    const int seg = blockIdx.x, ch = blockIdx.y;
    Aff<R> T;
    (void)scan_segment(p, sh, ch, seg, &T);
    if (threadIdx.x == 0) agg[(size_t)ch * gridDim.x + seg] = T;
}

// One warp per pair: boundary values, then the entering value of every segment
// as a warp scan over 32 segments at a time (lane s holds segment base + s).
template <typename R>
__global__ void __launch_bounds__(32) k_scan_segments(const KParams<R> p, const Aff<R> *__restrict__ agg,
                                                      r2<R> *__restrict__ enter, int nseg)
{
    IterState *st = p.st;
    if (*(volatile int *)&st->status != ST_RUNNING) return;
    const int lane = threadIdx.x & 31;
    const int fb = *(volatile int *)&st->base;
    const int J = p.J, P = p.P, pp = blockIdx.x;
    // mu < 0 enters through the right face: prescribed / vacuum data or (reflecting)
    // the previous iterate's mirror flux, copied into the face slot as the march does
    r2<R> x;
    if (p.bc_right == BC_REFLECT) {
        x = ld2(p.refl + pp);
        if (lane == 0) st2(p.faceM[fb] + (size_t)J * P + pp, x.x, x.y);
    } else {
        x = ld2(p.faceM[fb] + (size_t)J * P + pp);
    }
    for (int c = 0; c < 2; ++c) {
        const int ch = 2 * pp + c;
        if (c == 1) {
            if (p.bc_left == BC_REFLECT) {
                if (lane == 0) st2(p.faceP[fb] + pp, x.x, x.y);  // this sweep's mu < 0 flux at x = 0
            } else {
                x = ld2(p.faceP[fb] + pp);
            }
        }
        for (int s0 = 0; s0 < nseg; s0 += 32) {
            const int sg = s0 + lane;
            Aff<R> I = sg < nseg ? agg[(size_t)ch * nseg + sg] : aff_id<R>();
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const Aff<R> e = aff_shfl_up(I, d);
                if (lane >= d) I = aff_then(e, I);
            }
            Aff<R> E = aff_shfl_up(I, 1);
            if (lane == 0) E = aff_id<R>();
            if (sg < nseg)
                enter[(size_t)ch * nseg + sg] = r2<R>{E.a * x.x + (E.b * x.y + E.e), E.c * x.x + (E.d * x.y + E.f)};
            // all 32 maps of this pass (identity beyond nseg) applied to the entering value
            const R a = __shfl_sync(FULL, I.a, 31), b = __shfl_sync(FULL, I.b, 31), cc = __shfl_sync(FULL, I.c, 31);
            const R d = __shfl_sync(FULL, I.d, 31), e = __shfl_sync(FULL, I.e, 31), f = __shfl_sync(FULL, I.f, 31);
            x = r2<R>{a * x.x + (b * x.y + e), cc * x.x + (d * x.y + f)};
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const KParams<R> p, const r2<R> *__restrict__ enter)
{
    __shared__ ScanShared<R> sh;
    IterState *st = p.st;
    if (*(volatile int *)&st->status != ST_RUNNING) return;
    const int fb = *(volatile int *)&st->base;
    const int seg = blockIdx.x, ch = blockIdx.y, nseg = gridDim.x;
    const int J = p.J, P = p.P;
    const int pp = ch >> 1, dir = (ch & 1) ? 1 : -1;
    const Aff<R> E = scan_segment<R>(p, sh, ch, seg, nullptr);
    const r2<R> x0 = enter[(size_t)ch * nseg + seg];
    R xk = E.a * x0.x + (E.b * x0.y + E.e), xh = E.c * x0.x + (E.d * x0.y + E.f);
    const int s0 = seg * SCAN_SEG;
    const int n = J - s0 < SCAN_SEG ? J - s0 : SCAN_SEG;
    const R mu = ldg2(p.muw + pp).x;
    int mc = -1;
    r4<R> G{0, 0, 0, 0};
    for (int i = 0; i < SCAN_CPT; ++i) {
        const int k = threadIdx.x * SCAN_CPT + i;
        if (k >= n) break;
        const int m = sh.mat[k];
        if (m != mc) {
            mc = m;
            const Coef<R> c = load_coef(p.tab, m, P, pp);
            G = r4<R>{mu * c.pi, mu * c.ri, mu * c.ui, mu * c.vi};
        }
        const R nk = G.x * xk + (G.y * xh + sh.g[k].x);
        const R nh = G.z * xk + (G.w * xh + sh.g[k].y);
        xk = nk;
        xh = nh;
        const int j = dir > 0 ? s0 + k : J - 1 - (s0 + k);
        if (dir > 0) st2(p.faceP[fb] + (size_t)(j + 1) * P + pp, xk, xh);
        else st2(p.faceM[fb] + (size_t)j * P + pp, xk, xh);
    }
}

}  // namespace ocik
