// Backward-Euler (BE) variant of the OCI iteration (the paper's disabled
// section "Backward Euler transient implementation"): one time level per step,
// Sigma_hat = Sigma + 1/(v dt), the previous step's angular flux entering as a
// source psi^{n-1}/(v dt).  The cell is the SCB cell of the MB scheme without
// time moments: per ordinate pair, on the corner pair (L, R) as a complex
// number, A_{+mu} is multiplication by t = a - i mu/2 with
// a = (|mu| + dx Sigma)/2 + e (e = dx/(2 v dt)), A_{-mu} = conj(A_{+mu}), and
// the scattering coupling S = s (1 w^T) (s = dx Sigma_s/4) has the scalar
// capacitance K = 1/(1 - s m), m = sum_p 2 w_p Re(1/t_p).
// Source at the new time: Q_{k+1/2}; incident boundary data: its k+1/2 value.
// Storage shared with the MB path: faces carry the BE value in both slots and
// are read from .y (the k+1/2 slot, which holds the prescribed boundary value),
// psi_edge holds psi^n (+L, +R, -L, -R), phi the moments (L, R, L, R).
#pragma once
#include "oci_device.cuh"

namespace ocik {

template <typename R>
struct BeArgs {
    const r2<R> *tab;   // [n_mat][P]: 1/t (re, im)
    const double *K;    // [n_mat] scalar capacitance
    const float2 *Kf;   // [n_mat] the same as a double-float pair (FP32 path)
};

// One BE OCI iteration; one warp per cell, lanes over ordinate pairs.
template <typename R>
__global__ void __launch_bounds__(256) k_be_cells(const KParams<R> p, const BeArgs<R> be)
{
    int iter, base;
    if (!iteration_prologue(p, iter, base)) return;
    const int lane = threadIdx.x & 31;
    const int J = p.J, P = p.P;
    const int frd = (base + iter) & 1, fwr = frd ^ 1;
    const phi_t<R> *phr = iter == 0 ? p.phi0 : p.phi[iter & 1];
    phi_t<R> *phw = p.phi[(iter + 1) & 1];
    const r2<R> *fPr = p.faceP[frd], *fMr = p.faceM[frd];
    r2<R> *fPw = p.faceP[fwr], *fMw = p.faceM[fwr];
    const bool refl_l = p.bc_left == BC_REFLECT, refl_r = p.bc_right == BC_REFLECT;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    double d2 = 0.0, p2 = 0.0;
    float df2 = 0.f, pf2 = 0.f;  // FP32 path: per-thread partials in float, grid sums in double
    for (int cell = gw; cell < J; cell += nw) {
        const int m = p.mat[cell];
        const r4<R> qd = p.cellq[cell];
        const r2<R> es = p.matpar[m];
        // moment partials: double in FP64 mode; in FP32 mode float pairs summed
        // error-free across the warp (the FP64 pipe is slow on this GPU)
        R rLr = 0, rRr = 0;
        for (int pp = lane; pp < P; pp += 32) {
            const r2<R> mw = p.muw[pp];
            const r2<R> it = be.tab[(size_t)m * P + pp];
            const r4<R> pe = p.psi_edge[(size_t)cell * P + pp];
            const R inP = (refl_l && cell == 0) ? fMr[pp].y : fPr[(size_t)cell * P + pp].y;
            const R inM = (refl_r && cell == J - 1) ? fPr[(size_t)J * P + pp].y : fMr[(size_t)(cell + 1) * P + pp].y;
            // u = c+ ; v = conj(c-)
            const R ur = qd.z + es.x * pe.x + mw.x * inP, ui = qd.w + es.x * pe.y;
            const R vr = qd.z + es.x * pe.z, vi = -(qd.w + es.x * pe.w + mw.x * inM);
            const R yr = ur * it.x - ui * it.y, yi = ur * it.y + ui * it.x;
            const R zr = vr * it.x - vi * it.y, zi = vr * it.y + vi * it.x;
            rLr += mw.y * (yr + zr);
            rRr += mw.y * (yi - zi);
        }
        // phi = K r (double in FP64 mode, double-float in FP32 mode)
        double fL = 0.0, fR = 0.0;
        ff fLf{0.f, 0.f}, fRf{0.f, 0.f};
        R sL, sR;
        if constexpr (sizeof(R) == 8) {
            double rL = rLr, rR = rRr;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                rL += __shfl_xor_sync(FULL, rL, o);
                rR += __shfl_xor_sync(FULL, rR, o);
            }
            const double K = be.K[m];
            fL = K * rL;
            fR = K * rR;
            sL = (R)(es.y * fL);
            sR = (R)(es.y * fR);
        } else {
            ff aL{(float)rLr, 0.f}, aR{(float)rRr, 0.f};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                aL = ff_add(aL, ff{__shfl_xor_sync(FULL, aL.h, o), __shfl_xor_sync(FULL, aL.l, o)});
                aR = ff_add(aR, ff{__shfl_xor_sync(FULL, aR.h, o), __shfl_xor_sync(FULL, aR.l, o)});
            }
            const float2 K = be.Kf[m];
            fLf = ff_mul(ff{K.x, K.y}, aL);
            fRf = ff_mul(ff{K.x, K.y}, aR);
            sL = (R)(es.y * __fadd_rn(fLf.h, fLf.l));
            sR = (R)(es.y * __fadd_rn(fRf.h, fRf.l));
        }
        // outgoing corners: +mu R = Im(y + s phi/t), -mu L = Re(z + s conj(phi)/t)
        for (int pp = lane; pp < P; pp += 32) {
            const r2<R> mw = p.muw[pp];
            const r2<R> it = be.tab[(size_t)m * P + pp];
            const r4<R> pe = p.psi_edge[(size_t)cell * P + pp];
            const R inP = (refl_l && cell == 0) ? fMr[pp].y : fPr[(size_t)cell * P + pp].y;
            const R inM = (refl_r && cell == J - 1) ? fPr[(size_t)J * P + pp].y : fMr[(size_t)(cell + 1) * P + pp].y;
            const R ur = qd.z + es.x * pe.x + mw.x * inP, ui = qd.w + es.x * pe.y;
            const R vr = qd.z + es.x * pe.z, vi = -(qd.w + es.x * pe.w + mw.x * inM);
            const R yi = ur * it.y + ui * it.x, zr = vr * it.x - vi * it.y;
            const R outP = yi + (sL * it.y + sR * it.x);
            const R outM = zr + (sL * it.x + sR * it.y);
            fPw[(size_t)(cell + 1) * P + pp] = r2<R>{outP, outP};
            fMw[(size_t)cell * P + pp] = r2<R>{outM, outM};
        }
        if (lane < 4) {
            if constexpr (sizeof(R) == 8) {
                const double f = (lane & 1) ? fR : fL;
                if (lane < 2) {
                    const double d = f - PhiStore<R>::wide(phr[4 * (size_t)cell + lane]);
                    d2 += d * d;
                    p2 += f * f;
                }
                phw[4 * (size_t)cell + lane] = phi_from_double<R>(f);
            } else {
                const ff f = (lane & 1) ? fRf : fLf;
                if (lane < 2) {
                    const float2 old = phr[4 * (size_t)cell + lane];
                    const float d = ff_diff(f, ff{old.x, old.y});
                    df2 = __fmaf_rn(d, d, df2);
                    pf2 = __fmaf_rn(f.h, f.h, pf2);
                }
                phw[4 * (size_t)cell + lane] = make_float2(f.h, f.l);
            }
        }
    }
    finalize_iteration(d2 + (double)df2, p2 + (double)pf2, p.partials, p.st, p.cfg, iter, p.use_cond, p.cond);
}

// End of a BE step: if accepted, psi^n of every ordinate and corner from the
// last iteration's halo and moments goes to psi_edge, the next step's initial
// iterate (outgoing corners) to the free face buffer, phi to the published
// moments and to the next initial moments.
template <typename R>
__global__ void __launch_bounds__(256) k_be_commit(const KParams<R> p, const BeArgs<R> be)
{
    IterState *st = p.st;
    const int status = st->status, iter = st->iter, base = st->base;
    const bool go = iter >= 1 && (status == ST_CONVERGED || (status == ST_MAXITER && p.cfg->commit_unconverged));
    const int frd = (base + iter - 1) & 1, fgs = frd ^ 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->committed = go ? 1 : 0;
        st->base_next = go ? fgs : base;
    }
    if (!go) return;
    const phi_t<R> *ph = p.phi[iter & 1];
    const int lane = threadIdx.x & 31;
    const int J = p.J, P = p.P;
    const r2<R> *fPr = p.faceP[frd], *fMr = p.faceM[frd];
    const bool refl_l = p.bc_left == BC_REFLECT, refl_r = p.bc_right == BC_REFLECT;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int cell = gw; cell < J; cell += nw) {
        const int m = p.mat[cell];
        const r4<R> qd = p.cellq[cell];
        const r2<R> es = p.matpar[m];
        const double fL = PhiStore<R>::wide(__ldcg(ph + 4 * (size_t)cell));
        const double fR = PhiStore<R>::wide(__ldcg(ph + 4 * (size_t)cell + 1));
        const R sL = (R)(es.y * fL), sR = (R)(es.y * fR);
        for (int pp = lane; pp < P; pp += 32) {
            const r2<R> mw = p.muw[pp];
            const r2<R> it = be.tab[(size_t)m * P + pp];
            const r4<R> pe = p.psi_edge[(size_t)cell * P + pp];
            const R inP = (refl_l && cell == 0) ? fMr[pp].y : fPr[(size_t)cell * P + pp].y;
            const R inM = (refl_r && cell == J - 1) ? fPr[(size_t)J * P + pp].y : fMr[(size_t)(cell + 1) * P + pp].y;
            // psi+ = (c+ + s phi) / t ; conj(psi-) = (conj(c-) + s conj(phi)) / t
            const R ur = qd.z + es.x * pe.x + mw.x * inP + sL, ui = qd.w + es.x * pe.y + sR;
            const R vr = qd.z + es.x * pe.z + sL, vi = -(qd.w + es.x * pe.w + mw.x * inM) - sR;
            const R yr = ur * it.x - ui * it.y, yi = ur * it.y + ui * it.x;
            const R zr = vr * it.x - vi * it.y, zi = vr * it.y + vi * it.x;
            p.psi_edge[(size_t)cell * P + pp] = r4<R>{yr, yi, zr, -zi};
            p.faceP[fgs][(size_t)(cell + 1) * P + pp] = r2<R>{yi, yi};
            p.faceM[fgs][(size_t)cell * P + pp] = r2<R>{zr, zr};
        }
        if (lane < 4) {
            const double f = (lane & 1) ? fR : fL;
            p.phi_out[4 * (size_t)cell + lane] = f;
            p.phi0[4 * (size_t)cell + lane] = phi_from_double<R>(f);
        }
    }
}

}  // namespace ocik
