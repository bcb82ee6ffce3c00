// state_dev.cuh — device bodies of the FP64 prediction and of the pose
// matrices, shared by the single-stream kernels (state.cu) and the batched
// serving kernels (serve_kernels.cu).
//
// The FP64 prediction step (App. E.1 transition with the
// linearisation of App. E.1, Eq. statepropagation, App. E.2 split into the
// pose prior and the velocity conditional), on one block.
//
// Controls from the IMU window (reading R13): u_lin = R_mid mean(acc) + g,
// R_mid = Exp(w_m dt / 2) R; u_ang = (R_end w_end - w_prev) / dt with w_end
// the least-squares line through the gyro samples at the last sample time,
// R_end = Exp(w_m dt) R, w_m = R mean(gyro).  Velocity integration reads the
// printed (dt)^2 as dt (R12).  Error state (dt, dtheta, dv, dw) with the
// rotation error on the left (R14): A = diag(I, Exp(w dt)),
// B = diag(dt I, J_l(w dt) dt), F = [[A, B], [0, I]],
// Sigma' = F Sigma F^T + [[B Qv B^T + Qp, B Qv], [Qv B^T, Qv]].
// The kernel also starts the Gauss-Newton iterate at the prior mean.
#pragma once

#include "kernels.h"
#include "linalg64.cuh"
#include "prism_dev.cuh"

namespace prism {

// The prediction on one block of 256 threads.
__device__ __forceinline__ void predict_block(const KParams& P, DevState* dev, const double* __restrict__ imu,
                                              int n, double dt) {
    __shared__ double B[36], F[144], T1[144], Sig[144], Cv[144], Svp[36], Spv[36], Dm[36], Spp[36], Prec[36];
    __shared__ double Rw[9], Jl[9], vnew[6], Lch[36], rdg[6];
    __shared__ int ok;
    __shared__ double sums[8];   // mean t, acc (3), gyro (3), then t_end
    __shared__ double fit[4];    // sum dt^2, sum dt * dgyro (3)
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) dev->flags = 0;   // a new step: only its own kernels raise flags
    // the previous covariance, staged once (the products below read it in
    // dependent chains)
    for (int e = tid; e < 144; e += blockDim.x) Cv[e] = dev->cov[e];
    // IMU window statistics on warp 0: lane l takes samples l, l + 32, ...;
    // the warp reduction order is fixed, so the result is deterministic.
    if (tid < 32) {
        const double inv_n = n > 0 ? 1.0 / n : 0.0;
        double a[7] = {0, 0, 0, 0, 0, 0, 0}, te = -1e300;
        for (int i = lane; i < n; i += 32) {
            for (int c = 0; c < 7; ++c) a[c] += imu[7 * i + c];
            te = fmax(te, imu[7 * i]);
        }
        for (int c = 0; c < 7; ++c) {
            double v = a[c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            a[c] = v * inv_n;
        }
        for (int o = 16; o > 0; o >>= 1) te = fmax(te, __shfl_xor_sync(0xffffffffu, te, o));
        double f[4] = {0, 0, 0, 0};
        for (int i = lane; i < n; i += 32) {
            const double d = imu[7 * i] - a[0];
            f[0] = fma(d, d, f[0]);
            for (int c = 0; c < 3; ++c) f[1 + c] = fma(d, imu[7 * i + 4 + c] - a[4 + c], f[1 + c]);
        }
        for (int c = 0; c < 4; ++c) {
            double v = f[c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            f[c] = v;
        }
        if (lane == 0) {
            for (int c = 0; c < 7; ++c) sums[c] = a[c];
            sums[7] = te;
            for (int c = 0; c < 4; ++c) fit[c] = f[c];
        }
    }
    __syncthreads();
    // The controls and the mean propagation on warp 0, one entry a lane
    // (GB300's FP64 pipe is paced by warp instructions, not lanes).
    if (tid < 32) {
        if (lane == 0) ok = 1;
        double qm[4] = {dev->q[0], dev->q[1], dev->q[2], dev->q[3]};
        quat_normalise(qm);   // every lane, the same operations
        // R(qm) entry e on lane e < 9
        const double Re = quat_R_entry_rn(qm[0], qm[1], qm[2], qm[3], lane < 9 ? lane : 0);
        const double inv_dt = 1.0 / dt;
        double u = 0.0;   // lanes 0..2: u_lin, lanes 3..5: u_ang (zero without IMU samples)
        if (n > 0) {
            const double tm = sums[0], tend = sums[7];
            const double acc[3] = {sums[1], sums[2], sums[3]}, gyr[3] = {sums[4], sums[5], sums[6]};
            const double slope_scale = fit[0] > 0.0 ? (tend - tm) / fit[0] : 0.0;
            double gend[3];
            for (int a = 0; a < 3; ++a) gend[a] = fma(fit[1 + a], slope_scale, gyr[a]);
            // wm = R gyr (lane a < 3), then to every lane
            const int ra = lane < 3 ? lane : 0;
            const double wml = fdot3(__shfl_sync(0xffffffffu, Re, 3 * ra), gyr[0],
                                     __shfl_sync(0xffffffffu, Re, 3 * ra + 1), gyr[1],
                                     __shfl_sync(0xffffffffu, Re, 3 * ra + 2), gyr[2]);
            const double wm[3] = {__shfl_sync(0xffffffffu, wml, 0), __shfl_sync(0xffffffffu, wml, 1),
                                  __shfl_sync(0xffffffffu, wml, 2)};
            // Rh = Exp(dt wm / 2) entries on lanes 0..8, Rf = Exp(dt wm) on lanes 9..17
            const bool hf = lane < 9;
            const int e = lane < 9 ? lane : (lane < 18 ? lane - 9 : 0), ei = e / 3, ej = e % 3;
            double vrot[3];
            for (int a = 0; a < 3; ++a) vrot[a] = hf ? 0.5 * dt * wm[a] : dt * wm[a];
            const double Ee = so3_exp_jl_entry(vrot, true, ei, ej);
            // Rmid = Rh R on lanes 0..8, Rend = Rf R on lanes 9..17 (entry (i, j) a fdot3 over k)
            const int rb = hf ? 3 * ei : 9 + 3 * ei;
            const double Me = fdot3(__shfl_sync(0xffffffffu, Ee, rb), __shfl_sync(0xffffffffu, Re, ej),
                                    __shfl_sync(0xffffffffu, Ee, rb + 1), __shfl_sync(0xffffffffu, Re, 3 + ej),
                                    __shfl_sync(0xffffffffu, Ee, rb + 2), __shfl_sync(0xffffffffu, Re, 6 + ej));
            // am = Rmid acc on lanes 0..2, we = Rend gend on lanes 3..5
            const bool lin = lane < 3;
            const int rr = lane < 3 ? lane : (lane < 6 ? lane - 3 : 0);
            const int src = (lin ? 0 : 9) + 3 * rr;
            const double y = fdot3(__shfl_sync(0xffffffffu, Me, src), lin ? acc[0] : gend[0],
                                   __shfl_sync(0xffffffffu, Me, src + 1), lin ? acc[1] : gend[1],
                                   __shfl_sync(0xffffffffu, Me, src + 2), lin ? acc[2] : gend[2]);
            if (lane < 3) u = y + (lane == 2 ? -P.gravity : 0.0);
            else if (lane < 6) u = (y - dev->w[lane - 3]) * inv_dt;
        }
        // the new velocities (lanes 0..5) and position (lanes 0..2)
        double vn = 0.0;
        if (lane < 6) {
            const double vold = lane < 3 ? dev->v[lane] : dev->w[lane - 3];
            vn = fma(u, dt, vold);
            vnew[lane] = vn;
            if (lane < 3) {
                dev->pv[lane] = vn;
                dev->pt[lane] = fma(vn, dt, dev->t[lane]);
            } else {
                dev->pw[lane - 3] = vn;
            }
        }
        double wdt[3];
        for (int a = 0; a < 3; ++a) wdt[a] = __shfl_sync(0xffffffffu, vn, 3 + a) * dt;
        // Rw = Exp(wdt) entries on lanes 0..8, J_l(wdt) on lanes 9..17
        {
            const int e = lane < 9 ? lane : (lane < 18 ? lane - 9 : 0);
            const double v = so3_exp_jl_entry(wdt, lane < 9, e / 3, e % 3);
            if (lane < 9) Rw[lane] = v;
            else if (lane < 18) Jl[lane - 9] = v;
        }
        // the prior quaternion: normalise(quat_exp(wdt) (x) qm), component lane & 3
        const double qn = warp_quat_exp_mul(wdt, qm);
        if (lane < 4) dev->pq[lane] = qn;
    }
    __syncthreads();
    // A, B, F
    for (int e = tid; e < 144; e += blockDim.x) {
        int i = e / 12, j = e % 12;
        double f = 0.0;
        if (i < 6 && j < 6) {
            f = (i < 3 && j < 3) ? (i == j ? 1.0 : 0.0) : ((i >= 3 && j >= 3) ? Rw[3 * (i - 3) + j - 3] : 0.0);
        } else if (i < 6 && j >= 6) {
            int jj = j - 6;
            f = (i < 3 && jj < 3) ? (i == jj ? dt : 0.0)
                                  : ((i >= 3 && jj >= 3) ? Jl[3 * (i - 3) + jj - 3] * dt : 0.0);
            B[6 * i + jj] = f;
        } else if (i >= 6 && j >= 6) {
            f = (i == j) ? 1.0 : 0.0;
        }
        F[e] = f;
    }
    __syncthreads();
    block_matmul<12, 12, 12>(F, Cv, T1);
    block_matmul_nt<12, 12, 12>(T1, F, Sig);
    // transition noise
    for (int e = tid; e < 144; e += blockDim.x) {
        int i = e / 12, j = e % 12;
        auto qv = [&](int k) { double s = P.sigma_vel[k < 3 ? 0 : 1]; return s * s; };
        auto qp = [&](int k) { double s = P.sigma_pose[k < 3 ? 0 : 1]; return s * s; };
        double add = 0.0;
        if (i < 6 && j < 6) {
            for (int k = 0; k < 6; ++k) add = fma(B[6 * i + k] * qv(k), B[6 * j + k], add);
            if (i == j) add += qp(i);
        } else if (i < 6 && j >= 6) {
            add = B[6 * i + (j - 6)] * qv(j - 6);
        } else if (i >= 6 && j < 6) {
            add = B[6 * j + (i - 6)] * qv(i - 6);
        } else if (i == j) {
            add = qv(i - 6);
        }
        T1[e] = Sig[e] + add;
    }
    __syncthreads();
    for (int e = tid; e < 144; e += blockDim.x) {
        int i = e / 12, j = e % 12;
        double m = 0.5 * (T1[e] + T1[12 * j + i]);
        Sig[e] = m;
        dev->pcov[e] = m;
    }
    __syncthreads();
    for (int e = tid; e < 36; e += blockDim.x) {
        int i = e / 6, j = e % 6;
        dev->cov_pp[e] = Sig[12 * i + j];
        Spp[e] = Sig[12 * i + j];
        Spv[e] = Sig[12 * i + 6 + j];
        Svp[e] = Sig[12 * (6 + i) + j];
    }
    __syncthreads();
    if (!spd_inverse_block<6>(Spp, Prec, Lch, rdg, &ok)) {
        if (tid == 0) dev->flags |= FLAG_PRIOR_NOTPD;
        return;
    }
    block_matmul<6, 6, 6>(Svp, Prec, Dm);
    block_matmul<6, 6, 6>(Dm, Spv, T1);
    for (int e = tid; e < 36; e += blockDim.x) {
        int i = e / 6, j = e % 6;
        dev->prec_pp[e] = Prec[e];
        dev->D[e] = Dm[e];
        double a = Sig[12 * (6 + i) + 6 + j] - T1[e];
        double b = Sig[12 * (6 + j) + 6 + i] - T1[6 * j + i];
        dev->cov_vel[e] = 0.5 * (a + b);
    }
    if (tid < 6) dev->xi[tid] = 0.0;
    if (tid < 3) dev->cur_pose[tid] = dev->pt[tid];
    if (tid < 4) dev->cur_pose[3 + tid] = dev->pq[tid];
}

// FP32 decision matrices of a pose (see PrepKind), computed once per pose by
// the FP64 recipe so that no kernel block repeats the FP64 chain; for
// PREP_REL also the Gauss-Newton tangent map of the current iterate (see
// track_dev.cuh).  All 32 lanes of one warp call it; entries go one a lane.
__device__ __forceinline__ void prep_mats_warp(DevState* dev, int kind, const PoseArg& pose) {
    const int lane = threadIdx.x & 31;
    switch (kind) {
        case PREP_STATE:
            warp_mats_c2w(dev->t, dev->c2w);
            warp_mats_w2c(dev->t, dev->w2c);
            break;
        case PREP_AUX_C2W:
            warp_mats_c2w(pose.p, dev->aux);
            break;
        case PREP_AUX_REL:
            warp_mats_rel(pose.p, dev->anchor_pose, dev->aux);
            break;
        default: {
            // t[3] and q[4] are contiguous: the state mean's pose
            const double* anchor = kind == PREP_REL_NEXT ? dev->t : dev->anchor_pose;
            warp_mats_rel(dev->cur_pose, anchor, dev->rel);
            // Ra (lanes 0..8), then the prior's terms of the iterate in anchor-frame
            // coordinates
            const double* qa = anchor + 3;
            const double v = quat_R_entry_rn(qa[0], qa[1], qa[2], qa[3], lane < 9 ? lane : 0);
            __shared__ double s_ra[9], s_scr[69];
            if (lane < 9) {
                s_ra[lane] = v;
                dev->gn_Ci[lane] = v;
            }
            __syncwarp();
            warp_gn_prior_terms(s_ra, dev->prec_pp, dev->xi, dev->gn_Ci + 9, dev->gn_Lp, dev->gn_m, dev->gn_Ji,
                                s_scr);
            // the localisation's constants: q0 = conj(q_anchor) (x) q_prior on
            // lanes 24..27, b0 = Ra^T (t_prior - t_anchor) on lanes 28..30
            const int c = lane & 3;
            const double q0 = warp_quat_mul_component(c == 0 ? qa[0] : -qa[c], dev->pq);
            if (lane >= 24 && lane < 28) dev->gn_q0[c] = q0;
            const int i2 = lane >= 28 && lane < 31 ? lane - 28 : 0;
            const double rb0 = __shfl_sync(0xffffffffu, v, i2), rb1 = __shfl_sync(0xffffffffu, v, 3 + i2),
                         rb2 = __shfl_sync(0xffffffffu, v, 6 + i2);
            const double b0 = fdot3(rb0, dev->pt[0] - anchor[0], rb1, dev->pt[1] - anchor[1], rb2,
                                    dev->pt[2] - anchor[2]);
            if (lane >= 28 && lane < 31) dev->gn_b0[i2] = b0;
        }
    }
}

}  // namespace prism
