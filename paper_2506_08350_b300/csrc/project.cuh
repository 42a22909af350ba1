// Device-side projection of one Gaussian and its adjoint (FP32).
//
// Forward (Sec. 3): q -> R (unit quaternion, w first), Sigma = R S S^T R^T
// (Eq. gaussian_decompose, S = diag(exp(log_scale))), camera-space mean
// t = W x + tau, cull t_z < near_z, J = d(pixel)/d(t) at t with x/z, y/z
// clamped to +-clip * tan(fov/2), Sigma' = J W Sigma W^T J^T + dilation I
// (Eq. gaussian_projection), conic = Sigma'^-1, mu = (f_x t_x/t_z + c_x,
// f_y t_y/t_z + c_y), opacity = sigmoid(logit).
// Adjoint: reverse mode of the same chain (Supp. D.4 items 1-4).
#pragma once
#include "common.cuh"

namespace hcgs {

struct ProjArgs {
    int V, N, C, L, H, W;
    int tilesX, tilesY, ctX, ctY;
    float amin, amax, teps, dil, near_z, clip;
    int* status;  // device status word (device checks of the bounds-checked build)
    uint32_t M;   // bucket instances (once known)
};

inline ProjArgs make_proj_args(const hcgs_saved* s) {
    ProjArgs a;
    a.V = s->V; a.N = s->N; a.C = s->C; a.L = s->L; a.H = s->H; a.W = s->W;
    a.tilesX = s->tilesX; a.tilesY = s->tilesY; a.ctX = s->ctX; a.ctY = s->ctY;
    a.amin = s->opts.alpha_min; a.amax = s->opts.alpha_max; a.teps = s->opts.T_eps;
    a.dil = s->opts.cov2d_dilation; a.near_z = s->opts.near_z; a.clip = s->opts.clip_factor;
    a.status = nullptr;
    a.M = (uint32_t)s->M;
    return a;
}

// float4s per rasterizer record: (mu, A, B), (C, o, w0), (w1, w2), (w3, -)
__host__ __device__ inline int rec_count(int C) { return C <= 1 ? 2 : (C <= 3 ? 3 : 4); }
// floats per 2D gradient record: pixel moments of -dL/dpower 5, o dL/do 1, dL/dw 2C
__host__ __device__ inline int g2d_count(int C) { return 6 + 2 * C; }

struct ProjF {
    bool valid;
    float qn[4], qnorm, R[9], s[3], Sig[9];
    float t[3], tcx, tcy;
    int clx, cly;
    float J[6], T[6];
    float cov[3], conic[3];
    float2 mu;
    float o, depth;
};

// The view-independent factors of the 3D covariance: the normalised
// quaternion, its rotation R and the scales s = exp(log_scale).
__device__ __forceinline__ void sigma_factors(const float* ls, const float* q, ProjF& P) {
    const float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    P.qnorm = sqrtf(qq);
    for (int i = 0; i < 4; i++) P.qn[i] = q[i] / P.qnorm;
    const float w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
    P.R[0] = 1.f - 2.f * (y * y + z * z); P.R[1] = 2.f * (x * y - w * z); P.R[2] = 2.f * (x * z + w * y);
    P.R[3] = 2.f * (x * y + w * z); P.R[4] = 1.f - 2.f * (x * x + z * z); P.R[5] = 2.f * (y * z - w * x);
    P.R[6] = 2.f * (x * z - w * y); P.R[7] = 2.f * (y * z + w * x); P.R[8] = 1.f - 2.f * (x * x + y * y);
    for (int i = 0; i < 3; i++) P.s[i] = expf(ls[i]);
}

__device__ __forceinline__ void project_one(const ProjArgs& a, const float* mean, const float* ls, const float* q,
                                            float logit, const float* cam, ProjF& P) {
    const float* Vm = cam;
    const float fx = cam[16], fy = cam[17], cx = cam[18], cy = cam[19];
    for (int i = 0; i < 3; i++)
        P.t[i] = Vm[4 * i] * mean[0] + Vm[4 * i + 1] * mean[1] + Vm[4 * i + 2] * mean[2] + Vm[4 * i + 3];
    P.depth = P.t[2];
    P.valid = false;
    P.o = 1.f / (1.f + expf(-logit));
    P.mu = make_float2(0.f, 0.f);
    P.conic[0] = P.conic[1] = P.conic[2] = 0.f;
    P.cov[0] = P.cov[1] = P.cov[2] = 0.f;
    if (!(P.t[2] >= a.near_z)) return;
    sigma_factors(ls, q, P);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            float acc = 0.f;
            for (int k = 0; k < 3; k++) acc += P.R[3 * i + k] * P.s[k] * P.s[k] * P.R[3 * j + k];
            P.Sig[3 * i + j] = acc;
        }
    const float tz = P.t[2];
    P.tcx = P.t[0];
    P.tcy = P.t[1];
    P.clx = P.cly = 0;
    if (a.clip > 0.f) {
        const float limx = a.clip * (0.5f * a.W) / fx, limy = a.clip * (0.5f * a.H) / fy;
        const float rx = P.t[0] / tz, ry = P.t[1] / tz;
        if (rx > limx) { P.tcx = limx * tz; P.clx = 1; }
        else if (rx < -limx) { P.tcx = -limx * tz; P.clx = -1; }
        if (ry > limy) { P.tcy = limy * tz; P.cly = 1; }
        else if (ry < -limy) { P.tcy = -limy * tz; P.cly = -1; }
    }
    P.J[0] = fx / tz; P.J[1] = 0.f; P.J[2] = -fx * P.tcx / (tz * tz);
    P.J[3] = 0.f; P.J[4] = fy / tz; P.J[5] = -fy * P.tcy / (tz * tz);
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++) P.T[3 * i + j] = P.J[3 * i] * Vm[j] + P.J[3 * i + 1] * Vm[4 + j] + P.J[3 * i + 2] * Vm[8 + j];
    float TS[6];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++)
            TS[3 * i + j] = P.T[3 * i] * P.Sig[j] + P.T[3 * i + 1] * P.Sig[3 + j] + P.T[3 * i + 2] * P.Sig[6 + j];
    const float c00 = TS[0] * P.T[0] + TS[1] * P.T[1] + TS[2] * P.T[2];
    const float c01 = TS[0] * P.T[3] + TS[1] * P.T[4] + TS[2] * P.T[5];
    const float c11 = TS[3] * P.T[3] + TS[4] * P.T[4] + TS[5] * P.T[5];
    P.cov[0] = c00 + a.dil;
    P.cov[1] = c01;
    P.cov[2] = c11 + a.dil;
    const float det = P.cov[0] * P.cov[2] - P.cov[1] * P.cov[1];
    if (!(det > 0.f)) return;
    const float id = 1.f / det;
    P.conic[0] = P.cov[2] * id;
    P.conic[1] = -P.cov[1] * id;
    P.conic[2] = P.cov[0] * id;
    P.mu = make_float2(fx * P.t[0] / tz + cx, fy * P.t[1] / tz + cy);
    P.valid = true;
}

// One view's part of the projection adjoint: accumulates dL/dmean and
// dL/dSigma (the 3D covariance, 3 x 3) from dL/dmu and dL/d(A, B, C) of the
// conic (A, B; B, C), B counted once.  Sigma does not depend on the view, so
// its gradient is summed over the views and mapped to the log-scales and the
// rotation once (sigma_backward).
__device__ __forceinline__ void project_one_backward(const ProjArgs& a, const ProjF& P, const float* cam, float2 gmu,
                                                     float gA, float gB, float gC, float* gm, float* gsig) {
    const float* Vm = cam;
    const float fx = cam[16], fy = cam[17];
    // conic -> Sigma': G_S = -K G_K K with G_K = [[gA, gB/2], [gB/2, gC]]
    const float K0 = P.conic[0], K1 = P.conic[1], K2 = P.conic[2];
    const float g0 = gA, g1 = 0.5f * gB, g2 = gC;
    const float t00 = K0 * g0 + K1 * g1, t01 = K0 * g1 + K1 * g2;
    const float t10 = K1 * g0 + K2 * g1, t11 = K1 * g1 + K2 * g2;
    const float S00 = -(t00 * K0 + t01 * K1), S01 = -(t00 * K1 + t01 * K2);
    const float S10 = -(t10 * K0 + t11 * K1), S11 = -(t10 * K1 + t11 * K2);
    const float GS[4] = {S00, 0.5f * (S01 + S10), 0.5f * (S01 + S10), S11};
    // Sigma' = T Sigma T^T: dL/dSigma = T^T G T, dL/dT = 2 G T Sigma
    float GT[6];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            float acc = 0.f;
            for (int p = 0; p < 2; p++)
                for (int r = 0; r < 2; r++) acc += P.T[3 * p + i] * GS[2 * p + r] * P.T[3 * r + j];
            gsig[3 * i + j] += acc;
        }
    float TSig[6];
    for (int r = 0; r < 2; r++)
        for (int j = 0; j < 3; j++)
            TSig[3 * r + j] = P.T[3 * r] * P.Sig[j] + P.T[3 * r + 1] * P.Sig[3 + j] + P.T[3 * r + 2] * P.Sig[6 + j];
    for (int p = 0; p < 2; p++)
        for (int j = 0; j < 3; j++) GT[3 * p + j] = 2.f * (GS[2 * p] * TSig[j] + GS[2 * p + 1] * TSig[3 + j]);
    // T = J W3: dL/dJ = dL/dT W3^T
    float GJ[6];
    for (int p = 0; p < 2; p++)
        for (int k = 0; k < 3; k++) GJ[3 * p + k] = GT[3 * p] * Vm[4 * k] + GT[3 * p + 1] * Vm[4 * k + 1] + GT[3 * p + 2] * Vm[4 * k + 2];
    const float tx = P.t[0], ty = P.t[1], tz = P.t[2];
    const float iz = 1.f / tz, iz2 = iz * iz, iz3 = iz2 * iz;
    float gt0 = gmu.x * fx * iz;
    float gt1 = gmu.y * fy * iz;
    float gt2 = -gmu.x * fx * tx * iz2 - gmu.y * fy * ty * iz2;
    gt2 += -GJ[0] * fx * iz2 - GJ[4] * fy * iz2;
    if (P.clx == 0) { gt0 += -GJ[2] * fx * iz2; gt2 += GJ[2] * 2.f * fx * tx * iz3; }
    else            { gt2 += GJ[2] * fx * P.tcx * iz3; }
    if (P.cly == 0) { gt1 += -GJ[5] * fy * iz2; gt2 += GJ[5] * 2.f * fy * ty * iz3; }
    else            { gt2 += GJ[5] * fy * P.tcy * iz3; }
    for (int k = 0; k < 3; k++) gm[k] += Vm[k] * gt0 + Vm[4 + k] * gt1 + Vm[8 + k] * gt2;
}

// dL/d(log_scale, quat) from dL/dSigma (summed over the views), with the
// view-independent rotation and scales of P.
__device__ __forceinline__ void sigma_backward(const ProjF& P, const float* GSig, float* gls, float* gq) {
    // Sigma = M M^T, M = R diag(s): dL/dM = 2 GSig M
    float GR[9];
    for (int j = 0; j < 3; j++) {
        float gs = 0.f;
        for (int i = 0; i < 3; i++) {
            float gMij = 0.f;
            for (int k = 0; k < 3; k++) gMij += 2.f * GSig[3 * i + k] * P.R[3 * k + j] * P.s[j];
            GR[3 * i + j] = gMij * P.s[j];
            gs += gMij * P.R[3 * i + j];
        }
        gls[j] += gs * P.s[j];
    }
    const float w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
    float gqn[4];
    gqn[0] = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    gqn[1] = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] - 2.f * x * GR[8]);
    gqn[2] = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] - 2.f * y * GR[8]);
    gqn[3] = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] + x * GR[6] + y * GR[7]);
    float dot = 0.f;
    for (int k = 0; k < 4; k++) dot += P.qn[k] * gqn[k];
    for (int k = 0; k < 4; k++) gq[k] += (gqn[k] - P.qn[k] * dot) / P.qnorm;
}

}  // namespace hcgs
