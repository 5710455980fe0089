// Per-element and per-vertex arithmetic of the PBNG node update, shared by
// the direct kernels (pbng_kernels.cu), the ring-layout kernels
// (pbng_ring.cu) and the adjoint (pbng_adjoint.cu).  All of it is float32,
// formed relative to the rest state so that nothing cancels as F -> I.
#pragma once

#include "pbng_ff.cuh"
#include "pbng_internal.h"

namespace pbng {
namespace el {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }

__device__ __forceinline__ float det3(float a, float b, float c, float d, float e, float f, float g,
                                      float h, float i) {
    return a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
}

// u_j - u_i from stored pairs: (hi_j - hi_i) + (lo_j - lo_i).
template <bool COMP>
__device__ __forceinline__ float3 pair_diff(float4 hj, float4 lj, float3 uh, float3 ul) {
    float3 d = make_float3(hj.x - uh.x, hj.y - uh.y, hj.z - uh.z);
    if (COMP) {
        d.x += lj.x - ul.x;
        d.y += lj.y - ul.y;
        d.z += lj.z - ul.z;
    }
    return d;
}

// q holds column 0 of adj(M) for the symmetric 4x4 M = N - t I (upper
// triangle m00 .. m33); replace it with the column of adj(M) whose diagonal
// entry is largest in magnitude (adj(M) = -p'(t) q q^T is negative
// semidefinite, so its diagonal is -p'(t) q_k^2).  M is symmetric, so is
// adj(M): the other diagonal and off-diagonal cofactors, in registers.
__device__ __forceinline__ void adjugate_best_column(float m00, float m01, float m02, float m03, float m11, float m12,
                                                     float m13, float m22, float m23, float m33, float* q) {
    const float a11 = det3(m00, m02, m03, m02, m22, m23, m03, m23, m33);
    const float a22 = det3(m00, m01, m03, m01, m11, m13, m03, m13, m33);
    const float a33 = det3(m00, m01, m02, m01, m11, m12, m02, m12, m22);
    const float a12 = -det3(m00, m02, m03, m01, m12, m13, m03, m23, m33);
    const float a13 = det3(m00, m02, m03, m01, m12, m13, m02, m22, m23);
    const float a23 = -det3(m00, m01, m03, m01, m11, m13, m02, m12, m23);
    float best = -q[0];
    int kb = 0;
    if (-a11 > best) { best = -a11; kb = 1; }
    if (-a22 > best) { best = -a22; kb = 2; }
    if (-a33 > best) { kb = 3; }
    if (kb == 1) {
        q[0] = q[1]; q[1] = a11; q[2] = a12; q[3] = a13;
    } else if (kb == 2) {
        q[0] = q[2]; q[1] = a12; q[2] = a22; q[3] = a23;
    } else if (kb == 3) {
        q[0] = q[3]; q[1] = a13; q[2] = a23; q[3] = a33;
    }
}

// Rotation part of F = I + H for the corotated energy (Section "Constitutive
// Models", Eq. cor, with R the rotation of the polar decomposition in SO(3)),
// as the unit quaternion q = (w, x, y, z) times `scale`.
//
// Method (Horn 1987, "Closed-form solution of absolute orientation using unit
// quaternions"; the polar use follows Higham & Noferini 2016): R(q) maximises
// tr(R^T F) over rotations, which is the SO(3) polar factor (the smallest
// singular value takes the sign of det F).  tr(R(q)^T F) = q^T N q for a
// traceless symmetric 4x4 N built linearly from F, so q is the eigenvector of
// N's largest eigenvalue.  Its characteristic polynomial is
//   p(t) = t^4 - 2|F|^2 t^2 - 8 det(F) t + |F|^4 - 4|cof F|^2,
// whose largest root is found by Newton from the upper bound sqrt(3)|F|
// (monotone, because p is real-rooted; the quotient uses the fast
// approximate division, which Newton's own correction absorbs).  The
// eigenvector is a column of adj(N - t I), which is rank one; column 0 is
// used when it is well scaled (rotation angle up to about 120 degrees), else
// the column with the largest diagonal entry.  N - tI is built from H, so the
// vector part of q, and with it R - I = 2w[v]x + 2[v]x^2, keep relative
// accuracy as H -> 0.
__device__ __forceinline__ void polar_quaternion(const float* H, float n2, float c2, float J, float scale,
                                                 float* qo) {
    const float k0 = n2 * n2 - 4.0f * c2;
    const float n23 = 3.0f * n2;
    float t = n23 * rsqrtf(n23);
    // dprev starts as an assumed previous step of 3e-3 t, so that a first
    // step below 3e-5 t (already in the quadratic range near a simple root)
    // ends the iteration.
    float dp = 1.0f, dprev = 3e-3f * t;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
        const float t2 = t * t;
        const float p = ((t2 - 2.0f * n2) * t - 8.0f * J) * t + k0;
        dp = (4.0f * t2 - 4.0f * n2) * t - 8.0f * J;
        const float d = __fdividef(p, dp);
        t -= d;
        const float ad = fabsf(d);
        // Converged; or quadratic convergence has set in (this step is at most
        // 1/100 of the previous one) and the step is below 1e-4 t, so the
        // next one would be below float resolution.  Near a double root the
        // steps only halve, so the iteration goes on to the 2e-7 t test.
        if (!(ad > 2e-7f * t) || (ad <= 1e-4f * t && ad <= 0.01f * dprev)) break;
        dprev = ad;
    }
    const float trH = H[0] + H[4] + H[8];
    const float m00 = (3.0f - t) + trH;
    const float m11 = (-1.0f - t) + (H[0] - H[4] - H[8]);
    const float m22 = (-1.0f - t) + (H[4] - H[0] - H[8]);
    const float m33 = (-1.0f - t) + (H[8] - H[0] - H[4]);
    const float m01 = H[7] - H[5], m02 = H[2] - H[6], m03 = H[3] - H[1];
    const float m12 = H[1] + H[3], m13 = H[2] + H[6], m23 = H[5] + H[7];
    // Column 0 of adj(M) = (+min00, -min01, +min02, -min03), the minors of
    // rows 1..3.  Expand each along row 1 with the six 2x2 minors of rows 2, 3
    // (columns a < b), which the four determinants share.
    const float k01 = m02 * m13 - m12 * m03, k02 = m02 * m23 - m22 * m03, k03 = m02 * m33 - m23 * m03;
    const float k12 = m12 * m23 - m22 * m13, k13 = m12 * m33 - m23 * m13, k23 = m22 * m33 - m23 * m23;
    float q[4];
    q[0] = m11 * k23 - m12 * k13 + m13 * k12;
    q[1] = -(m01 * k23 - m12 * k03 + m13 * k02);
    q[2] = m01 * k13 - m11 * k03 + m13 * k01;
    q[3] = -(m01 * k12 - m11 * k02 + m12 * k01);
    // adj(M) = -p'(t) q q^T, so q_0^2 = -adj_00 / p'(t).  Beyond about 120
    // degrees column 0 is poorly scaled: take the column of adj(M) with the
    // largest diagonal entry instead.
    if (!(-q[0] > 0.25f * dp)) adjugate_best_column(m00, m01, m02, m03, m11, m12, m13, m22, m23, m33, q);
    const float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (qq > 1e-30f && qq < 3.0e38f) {
        const float inv = scale * rsqrtf(qq);
#pragma unroll
        for (int k = 0; k < 4; ++k) qo[k] = q[k] * inv;
    } else {
        qo[0] = scale;
        qo[1] = qo[2] = qo[3] = 0.0f;
    }
}

// R - I (row major) of the rotation of F = I + H: 2 w [v]x + 2 (v v^T - |v|^2 I).
__device__ __forceinline__ void rotation_minus_identity(const float* H, float n2, float c2, float J,
                                                        float* RmI) {
    float q[4];
    polar_quaternion(H, n2, c2, J, 1.0f, q);
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
    RmI[0] = -2.0f * (yy + zz);
    RmI[1] = 2.0f * (xy - wz);
    RmI[2] = 2.0f * (xz + wy);
    RmI[3] = 2.0f * (xy + wz);
    RmI[4] = -2.0f * (xx + zz);
    RmI[5] = 2.0f * (yz - wx);
    RmI[6] = 2.0f * (xz - wy);
    RmI[7] = 2.0f * (yz + wx);
    RmI[8] = -2.0f * (xx + yy);
}

// Contribution of one incident tetrahedron to the force r and modified
// Hessian A (upper triangle a00 a01 a02 a11 a12 a22) of vertex i:
//   r -= V P(F) g_i,  A += V (2 mu |g_i|^2 I + lambda w w^T),  w = cof(F) g_i
// with F = I + sum_{j != i} (u_j - u_i) g_j^T and g_i = -(g_j1 + g_j2 + g_j3).
// A is Eq. mod_hess_dens for every model (Section "Lame Coefficients").
// gk = dN_jk/dX of the other three vertices, a = 2 mu V, b = lambda V,
// dk = u_jk - u_i.  P (Section "Constitutive Models"), with C = cof F and
// H = F - I:
//   kCorotated (Eq. cor)  V P g = a (H - (R - I)) g + b (J - 1) w
//   kNeoHookean (Eq. nh, lambda_hat = mu + lambda):
//     P = mu (F - C) + lambda_hat (J - 1) C,
//     V P g = (a/2) (F - C) g + (a/2 + b) (J - 1) w
//   kStableNeoHookean (Eq. snh with lambda on the volume term and the Lame
//     reparametrisation mu' = 4 mu / 3, lambda' = lambda + 5 mu / 6,
//     alpha = 1 + 3 mu' / (4 lambda') that makes its Hessian at F = I the
//     linear-elasticity one):
//     P = (3 mu'/4) (F - C) + mu' (I_C - 3) / (4 (1 + I_C)) F + lambda' (J - 1) C,
//     V P g = (a/2) (F - C) g + (a/6) (I_C - 3) / (1 + I_C) F g + (b + 5a/12) (J - 1) w
// where F - C = H + H^T - tr(H) I - cof(H) and I_C - 3 = 2 tr H + |H|^2 are
// formed from H, so the Neo-Hookean stresses keep relative accuracy at rest.
// Everything is written with s = g_j1 + g_j2 + g_j3 = -g_i: r gains
// +V P(F) s, and w = -cof(F) s enters A squared.  The corotated rotation
// acts on s through its quaternion (w, v) scaled by sqrt(2):
// (R - I) s = w (v x s) + v (v . s) - |v|^2 s.
// ACC adds to r and A; otherwise it overwrites them.
enum { kCorotated = 0, kNeoHookean = 1, kStableNeoHookean = 2 };

template <bool NEED_A, int MODEL, bool ACC = true>
__device__ __forceinline__ void element_math_m(float3 gj1, float3 gj2, float3 gj3, float a, float b,
                                               float3 d1, float3 d2, float3 d3, float* r, float* A) {
    const float g1[3] = {gj1.x, gj1.y, gj1.z}, g2[3] = {gj2.x, gj2.y, gj2.z}, g3[3] = {gj3.x, gj3.y, gj3.z};
    const float dd1[3] = {d1.x, d1.y, d1.z}, dd2[3] = {d2.x, d2.y, d2.z}, dd3[3] = {d3.x, d3.y, d3.z};
    float H[9];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) H[3 * p + q] = dd1[p] * g1[q] + dd2[p] * g2[q] + dd3[p] * g3[q];
    const float s[3] = {g1[0] + g2[0] + g3[0], g1[1] + g2[1] + g3[1], g1[2] + g2[2] + g3[2]};

    const float F0 = 1.0f + H[0], F4 = 1.0f + H[4], F8 = 1.0f + H[8];
    const float F1 = H[1], F2 = H[2], F3 = H[3], F5 = H[5], F6 = H[6], F7 = H[7];
    float C[9];
    C[0] = F4 * F8 - F5 * F7;
    C[1] = F5 * F6 - F3 * F8;
    C[2] = F3 * F7 - F4 * F6;
    C[3] = F7 * F2 - F8 * F1;
    C[4] = F8 * F0 - F6 * F2;
    C[5] = F6 * F1 - F7 * F0;
    C[6] = F1 * F5 - F2 * F4;
    C[7] = F2 * F3 - F0 * F5;
    C[8] = F0 * F4 - F1 * F3;
    // J - 1 = tr H + (sum of principal 2x2 minors of H) + det H.
    const float trH = H[0] + H[4] + H[8];
    const float Jm1 = trH + (H[0] * H[4] - H[1] * H[3] + H[0] * H[8] - H[2] * H[6] + H[4] * H[8] - H[5] * H[7]) +
                      det3(H[0], H[1], H[2], H[3], H[4], H[5], H[6], H[7], H[8]);
    float ws[3], Hs[3];  // cof(F) s = -w, H s
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        ws[p] = C[3 * p] * s[0] + C[3 * p + 1] * s[1] + C[3 * p + 2] * s[2];
        Hs[p] = H[3 * p] * s[0] + H[3 * p + 1] * s[1] + H[3 * p + 2] * s[2];
    }
    float f[3];  // V P(F) s
    const float bJ = b * Jm1;
    if (MODEL == kCorotated) {
        float n2 = 0.0f, c2 = 0.0f;
        const float Fm[9] = {F0, F1, F2, F3, F4, F5, F6, F7, F8};
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            n2 += Fm[k] * Fm[k];
            c2 += C[k] * C[k];
        }
        float q[4];
        polar_quaternion(H, n2, c2, 1.0f + Jm1, 1.41421356237309505f, q);
        const float x = q[1], y = q[2], z = q[3];
        const float cr[3] = {y * s[2] - z * s[1], z * s[0] - x * s[2], x * s[1] - y * s[0]};
        const float vs = x * s[0] + y * s[1] + z * s[2];
        const float vv = x * x + y * y + z * z;
        const float vq[3] = {x, y, z};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float rs = q[0] * cr[p] + (vq[p] * vs - vv * s[p]);
            f[p] = a * (Hs[p] - rs) + bJ * ws[p];
        }
    } else {
        // cof(H), then (F - C) s = H s + H^T s - tr(H) s - cof(H) s
        float K[9];
        K[0] = H[4] * H[8] - H[5] * H[7];
        K[1] = H[5] * H[6] - H[3] * H[8];
        K[2] = H[3] * H[7] - H[4] * H[6];
        K[3] = H[7] * H[2] - H[8] * H[1];
        K[4] = H[8] * H[0] - H[6] * H[2];
        K[5] = H[6] * H[1] - H[7] * H[0];
        K[6] = H[1] * H[5] - H[2] * H[4];
        K[7] = H[2] * H[3] - H[0] * H[5];
        K[8] = H[0] * H[4] - H[1] * H[3];
        const float ha = 0.5f * a;
        float qs = 0.0f, kv = ha + b;
        if (MODEL == kStableNeoHookean) {
            float hh = 0.0f;
#pragma unroll
            for (int k = 0; k < 9; ++k) hh += H[k] * H[k];
            const float ic3 = 2.0f * trH + hh;                  // I_C - 3
            qs = (a * (1.0f / 6.0f)) * __fdividef(ic3, 4.0f + ic3);
            kv = b + a * (5.0f / 12.0f);
        }
        const float kJ = kv * Jm1;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float Hts = H[p] * s[0] + H[3 + p] * s[1] + H[6 + p] * s[2];
            const float Ks = K[3 * p] * s[0] + K[3 * p + 1] * s[1] + K[3 * p + 2] * s[2];
            const float fcs = (Hs[p] + Hts) - trH * s[p] - Ks;
            float t = ha * fcs + kJ * ws[p];
            if (MODEL == kStableNeoHookean) t += qs * (s[p] + Hs[p]);
            f[p] = t;
        }
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) r[p] = ACC ? r[p] + f[p] : f[p];
    if (NEED_A) {
        const float ag = a * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
        const float bw0 = b * ws[0], bw1 = b * ws[1], bw2 = b * ws[2];
        const float e[6] = {ag + bw0 * ws[0], bw0 * ws[1], bw0 * ws[2], ag + bw1 * ws[1], bw1 * ws[2], ag + bw2 * ws[2]};
#pragma unroll
        for (int k = 0; k < 6; ++k) A[k] = ACC ? A[k] + e[k] : e[k];
    }
}

// The float32 companions of the extended-precision force (pbng_ff.cuh): the
// modified Hessian of Eq. mod_hess_dens, A = V (2 mu |g_i|^2 I + lambda w w^T)
// with w = cof(F) g_i (upper triangle, overwritten), and the quaternion
// estimate of the corotated polar rotation (scale 1) that the float-float
// force refines.  Same operands as element_math_m.
template <bool NEED_A, bool NEED_Q>
__device__ __forceinline__ void element_fp32_parts(float3 gj1, float3 gj2, float3 gj3, float a, float b, float3 d1,
                                                   float3 d2, float3 d3, float* A, float* q) {
    const float g1[3] = {gj1.x, gj1.y, gj1.z}, g2[3] = {gj2.x, gj2.y, gj2.z}, g3[3] = {gj3.x, gj3.y, gj3.z};
    const float dd1[3] = {d1.x, d1.y, d1.z}, dd2[3] = {d2.x, d2.y, d2.z}, dd3[3] = {d3.x, d3.y, d3.z};
    float H[9];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int c = 0; c < 3; ++c) H[3 * p + c] = dd1[p] * g1[c] + dd2[p] * g2[c] + dd3[p] * g3[c];
    const float F0 = 1.0f + H[0], F4 = 1.0f + H[4], F8 = 1.0f + H[8];
    const float F1 = H[1], F2 = H[2], F3 = H[3], F5 = H[5], F6 = H[6], F7 = H[7];
    float C[9];
    C[0] = F4 * F8 - F5 * F7;
    C[1] = F5 * F6 - F3 * F8;
    C[2] = F3 * F7 - F4 * F6;
    C[3] = F7 * F2 - F8 * F1;
    C[4] = F8 * F0 - F6 * F2;
    C[5] = F6 * F1 - F7 * F0;
    C[6] = F1 * F5 - F2 * F4;
    C[7] = F2 * F3 - F0 * F5;
    C[8] = F0 * F4 - F1 * F3;
    if (NEED_A) {
        const float s[3] = {g1[0] + g2[0] + g3[0], g1[1] + g2[1] + g3[1], g1[2] + g2[2] + g3[2]};
        float ws[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) ws[p] = C[3 * p] * s[0] + C[3 * p + 1] * s[1] + C[3 * p + 2] * s[2];
        const float ag = a * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
        const float bw0 = b * ws[0], bw1 = b * ws[1], bw2 = b * ws[2];
        A[0] = ag + bw0 * ws[0];
        A[1] = bw0 * ws[1];
        A[2] = bw0 * ws[2];
        A[3] = ag + bw1 * ws[1];
        A[4] = bw1 * ws[2];
        A[5] = ag + bw2 * ws[2];
    }
    if (NEED_Q) {
        const float trH = H[0] + H[4] + H[8];
        const float Jm1 = trH + (H[0] * H[4] - H[1] * H[3] + H[0] * H[8] - H[2] * H[6] + H[4] * H[8] - H[5] * H[7]) +
                          det3(H[0], H[1], H[2], H[3], H[4], H[5], H[6], H[7], H[8]);
        const float Fm[9] = {F0, F1, F2, F3, F4, F5, F6, F7, F8};
        float n2 = 0.0f, c2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            n2 += Fm[k] * Fm[k];
            c2 += C[k] * C[k];
        }
        polar_quaternion(H, n2, c2, 1.0f + Jm1, 1.0f, q);
    }
}

// The model is uniform over a launch (PassParams::model): one branch per call.
template <bool NEED_A>
__device__ __forceinline__ void element_math(int model, float3 gj1, float3 gj2, float3 gj3, float a, float b,
                                             float3 d1, float3 d2, float3 d3, float* r, float* A) {
    if (model == kNeoHookean)
        element_math_m<NEED_A, kNeoHookean>(gj1, gj2, gj3, a, b, d1, d2, d3, r, A);
    else if (model == kStableNeoHookean)
        element_math_m<NEED_A, kStableNeoHookean>(gj1, gj2, gj3, a, b, d1, d2, d3, r, A);
    else
        element_math_m<NEED_A, kCorotated>(gj1, gj2, gj3, a, b, d1, d2, d3, r, A);
}

// Body force, weak springs and plane contact of a vertex at displacement
// uh + ul (Section "Weak Constraints"), from its aux records
// x0 = (f^ext, K), x1 = (spring target displacement, n.X - d):
// r += f^ext; r -= K (u - t_u), A += K I; if s = n.X - d + n.u < 0:
// r -= k s n, A += k n n^T.
template <bool COMP, bool NEED_A>
__device__ __forceinline__ void vertex_terms(const DeviceMesh& m, float4 x0, float4 x1, float3 uh,
                                             float3 ul, float* r, float* A) {
    r[0] += x0.x;
    r[1] += x0.y;
    r[2] += x0.z;
    if (x0.w != 0.0f) {
        float e0 = uh.x - x1.x, e1 = uh.y - x1.y, e2 = uh.z - x1.z;
        if (COMP) { e0 += ul.x; e1 += ul.y; e2 += ul.z; }
        r[0] -= x0.w * e0;
        r[1] -= x0.w * e1;
        r[2] -= x0.w * e2;
        if (NEED_A) { A[0] += x0.w; A[3] += x0.w; A[5] += x0.w; }
    }
    if (m.k_contact > 0.0f) {
        float sd = x1.w + (m.pn_x * uh.x + m.pn_y * uh.y + m.pn_z * uh.z);
        if (COMP) sd += m.pn_x * ul.x + m.pn_y * ul.y + m.pn_z * ul.z;
        if (sd < 0.0f) {
            const float ks = m.k_contact * sd;
            r[0] -= ks * m.pn_x;
            r[1] -= ks * m.pn_y;
            r[2] -= ks * m.pn_z;
            if (NEED_A) {
                A[0] += m.k_contact * m.pn_x * m.pn_x;
                A[1] += m.k_contact * m.pn_x * m.pn_y;
                A[2] += m.k_contact * m.pn_x * m.pn_z;
                A[3] += m.k_contact * m.pn_y * m.pn_y;
                A[4] += m.k_contact * m.pn_y * m.pn_z;
                A[5] += m.k_contact * m.pn_z * m.pn_z;
            }
        }
    }
}

// The same vertex terms added to a float-float force r (residuals and the
// extended-precision passes): f^ext, and the spring and contact forces
// formed from the float-pair displacement (u - t by TwoSum).  The contact
// test is taken in float.
template <bool NEED_A>
__device__ __forceinline__ void vertex_terms_ff(const DeviceMesh& m, int v, float4 x0, float4 x1, float3 uh,
                                                float3 ul, ff::F2* r, float* A) {
    r[0] = ff::add(r[0], x0.x);
    r[1] = ff::add(r[1], x0.y);
    r[2] = ff::add(r[2], x0.z);
    if (m.aux_lo) {  // the low words of f^ext
        const float4 xl = m.aux_lo[v];
        r[0] = ff::add(r[0], xl.x);
        r[1] = ff::add(r[1], xl.y);
        r[2] = ff::add(r[2], xl.z);
    }
    if (x0.w != 0.0f) {
        const ff::F2 e0 = ff::add(ff::two_sum(uh.x, -x1.x), ul.x);
        const ff::F2 e1 = ff::add(ff::two_sum(uh.y, -x1.y), ul.y);
        const ff::F2 e2 = ff::add(ff::two_sum(uh.z, -x1.z), ul.z);
        r[0] = ff::sub(r[0], ff::mul(e0, x0.w));
        r[1] = ff::sub(r[1], ff::mul(e1, x0.w));
        r[2] = ff::sub(r[2], ff::mul(e2, x0.w));
        if (NEED_A) { A[0] += x0.w; A[3] += x0.w; A[5] += x0.w; }
    }
    if (m.k_contact > 0.0f) {
        const float sdf = x1.w + (m.pn_x * (uh.x + ul.x) + m.pn_y * (uh.y + ul.y) + m.pn_z * (uh.z + ul.z));
        if (sdf < 0.0f) {
            // gap n.X - d + n.u with the products exact
            ff::F2 sd = ff::mk(x1.w);
            sd = ff::add(sd, ff::two_prod(m.pn_x, uh.x));
            sd = ff::add(sd, ff::two_prod(m.pn_y, uh.y));
            sd = ff::add(sd, ff::two_prod(m.pn_z, uh.z));
            sd = ff::add(sd, m.pn_x * ul.x + m.pn_y * ul.y + m.pn_z * ul.z);
            const ff::F2 ks = ff::mul(sd, m.k_contact);
            r[0] = ff::sub(r[0], ff::mul(ks, m.pn_x));
            r[1] = ff::sub(r[1], ff::mul(ks, m.pn_y));
            r[2] = ff::sub(r[2], ff::mul(ks, m.pn_z));
            if (NEED_A) {
                A[0] += m.k_contact * m.pn_x * m.pn_x;
                A[1] += m.k_contact * m.pn_x * m.pn_y;
                A[2] += m.k_contact * m.pn_x * m.pn_z;
                A[3] += m.k_contact * m.pn_y * m.pn_y;
                A[4] += m.k_contact * m.pn_y * m.pn_z;
                A[5] += m.k_contact * m.pn_z * m.pn_z;
            }
        }
    }
}

// General weak constraints of Section "Weak Constraints" on free vertex v:
// for each constraint c with own coefficient beta (w0 - w1 at v),
// C = C0 + sum_q b_q u_q, r -= beta K C and A += beta^2 K (the second term
// of Eq. mod_hess).  The other vertices of c have other colours, so none of
// them is written by the pass that updates v.
// C is small next to the displacements it is formed from (a stiff binding
// holds its two points together), so it is accumulated without rounding
// loss: each b_q u_q as an exact product pair (FMA), summed with TwoSum, on
// top of the float-pair rest value C0.
__device__ __forceinline__ void acc_exact(float& s, float& c, float b, float u) {
    const float p = b * u;
    const float pe = __fmaf_rn(b, u, -p);  // b u - p exactly
    const float t = __fadd_rn(s, p);
    const float bp = __fadd_rn(t, -s);
    c += __fadd_rn(__fadd_rn(s, -__fadd_rn(t, -bp)), __fadd_rn(p, -bp)) + pe;
    s = t;
}

template <bool COMP, bool NEED_A>
__device__ __forceinline__ void weak_terms(const DeviceMesh& m, const State& s, int v, float* r, float* A) {
    if (!m.wc_off) return;
    const int k1 = m.wc_off[v + 1];
    for (int k = m.wc_off[v]; k < k1; ++k) {
        const int2 e = m.wc_list[k];
        const int c = e.x;
        const float beta = __int_as_float(e.y);
        const float4 c0 = m.wc_c0[2 * c], c0l = m.wc_c0[2 * c + 1];
        float S[3] = {c0.x, c0.y, c0.z}, E[3] = {c0l.x, c0l.y, c0l.z};
        for (int q = 0; q < 8; ++q) {
            const int j = m.wc_v[8 * c + q];
            if (j < 0) break;
            const float bq = m.wc_b[8 * c + q];
            const float4 h = s.hi[j];
            acc_exact(S[0], E[0], bq, h.x);
            acc_exact(S[1], E[1], bq, h.y);
            acc_exact(S[2], E[2], bq, h.z);
            if (COMP) {
                const float4 l = s.lo[j];
                E[0] += bq * l.x;
                E[1] += bq * l.y;
                E[2] += bq * l.z;
            }
        }
        const float C[3] = {S[0] + E[0], S[1] + E[1], S[2] + E[2]};
        const float* K = m.wc_k + 6 * c;
        const float KC0 = K[0] * C[0] + K[1] * C[1] + K[2] * C[2];
        const float KC1 = K[1] * C[0] + K[3] * C[1] + K[4] * C[2];
        const float KC2 = K[2] * C[0] + K[4] * C[1] + K[5] * C[2];
        r[0] -= beta * KC0;
        r[1] -= beta * KC1;
        r[2] -= beta * KC2;
        if (NEED_A) {
            const float b2 = beta * beta;
#pragma unroll
            for (int t = 0; t < 6; ++t) A[t] += b2 * K[t];
        }
    }
}

// The weak-constraint terms added to a float-float force r: C as the float
// pair S + E of the error-free accumulation above, K C and beta K C in
// float-float.
template <bool COMP, bool NEED_A>
__device__ __forceinline__ void weak_terms_ff(const DeviceMesh& m, const State& s, int v, ff::F2* r, float* A) {
    if (!m.wc_off) return;
    const int k1 = m.wc_off[v + 1];
    for (int k = m.wc_off[v]; k < k1; ++k) {
        const int2 e = m.wc_list[k];
        const int c = e.x;
        const float beta = __int_as_float(e.y);
        const float4 c0 = m.wc_c0[2 * c], c0l = m.wc_c0[2 * c + 1];
        float S[3] = {c0.x, c0.y, c0.z}, E[3] = {c0l.x, c0l.y, c0l.z};
        for (int q = 0; q < 8; ++q) {
            const int j = m.wc_v[8 * c + q];
            if (j < 0) break;
            const float bq = m.wc_b[8 * c + q];
            const float4 h = s.hi[j];
            acc_exact(S[0], E[0], bq, h.x);
            acc_exact(S[1], E[1], bq, h.y);
            acc_exact(S[2], E[2], bq, h.z);
            if (COMP) {
                const float4 l = s.lo[j];
                E[0] += bq * l.x;
                E[1] += bq * l.y;
                E[2] += bq * l.z;
            }
        }
        const ff::F2 C[3] = {ff::two_sum(S[0], E[0]), ff::two_sum(S[1], E[1]), ff::two_sum(S[2], E[2])};
        const float* K = m.wc_k + 6 * c;
        const int kk[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const ff::F2 KC = ff::add(ff::add(ff::mul(C[0], K[kk[p][0]]), ff::mul(C[1], K[kk[p][1]])),
                                      ff::mul(C[2], K[kk[p][2]]));
            r[p] = ff::sub(r[p], ff::mul(KC, beta));
        }
        if (NEED_A) {
            const float b2 = beta * beta;
#pragma unroll
            for (int t = 0; t < 6; ++t) A[t] += b2 * K[t];
        }
    }
}

// hi + lo += d, keeping the pair normalised (TwoSum, then Fast2Sum).
__device__ __forceinline__ void pair_add(float& hi, float& lo, float d) {
    const float s = __fadd_rn(hi, d);
    const float bp = __fadd_rn(s, -hi);
    const float e = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bp)), __fadd_rn(d, -bp));
    const float t = __fadd_rn(e, lo);
    const float h2 = __fadd_rn(s, t);
    lo = __fadd_rn(t, -__fadd_rn(h2, -s));
    hi = h2;
}

template <int W>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off, W);
    return v;
}

// The same W-lane sum in float-float arithmetic (the residual's vertex sums:
// their terms are far larger than the sum near an equilibrium): the high
// words are summed by TwoSum, their rounding errors and the low words in a
// float (Ogita, Rump and Oishi's Sum2), normalised once at the end.
template <int W>
__device__ __forceinline__ ff::F2 group_sum_ff(ff::F2 v) {
    float h = v.h, e = v.l;
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        const float ho = __shfl_xor_sync(kFull, h, off, W), eo = __shfl_xor_sync(kFull, e, off, W);
        const ff::F2 t = ff::two_sum(h, ho);
        h = t.h;
        e = ff::fadd(e, ff::fadd(eo, t.l));
    }
    return ff::quick_two_sum(h, e);
}

// |r|^2 of a float-float force in FP64.
__device__ __forceinline__ double norm2_ff(const ff::F2* r) {
    double q = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double v = ff::to_d(r[k]);
        q += v * v;
    }
    return q;
}

// Eq. pbgn_dx / pbgn_update: Delta = step A^{-1} r (adjugate; A is SPD by
// construction, Eq. mod_hess) and u_v += Delta in place.
template <bool COMP>
__device__ __forceinline__ void solve_and_write(State s, int v, float3 uh, float3 ul, const float* r,
                                                const float* A, PassParams pp, int32_t* err) {
    if (pp.skip_tol > 0.0f && r[0] * r[0] + r[1] * r[1] + r[2] * r[2] <= pp.skip_tol * pp.skip_tol) return;
    const float c00 = A[3] * A[5] - A[4] * A[4];
    const float c01 = A[2] * A[4] - A[1] * A[5];
    const float c02 = A[1] * A[4] - A[2] * A[3];
    const float c11 = A[0] * A[5] - A[2] * A[2];
    const float c12 = A[1] * A[2] - A[0] * A[4];
    const float c22 = A[0] * A[3] - A[1] * A[1];
    const float det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(det > 0.0f) || !(det < 3.0e38f)) {
        atomicOr(err, kErrNonSPD);
        return;
    }
    const float sc = __fdividef(pp.step, det);
    const float dx = sc * (c00 * r[0] + c01 * r[1] + c02 * r[2]);
    const float dy = sc * (c01 * r[0] + c11 * r[1] + c12 * r[2]);
    const float dz = sc * (c02 * r[0] + c12 * r[1] + c22 * r[2]);
    if (!(fabsf(dx) + fabsf(dy) + fabsf(dz) < 3.0e38f)) {  // NaN or infinity
        atomicOr(err, kErrNonFinite);
        return;
    }
    if (COMP) {
        pair_add(uh.x, ul.x, dx);
        pair_add(uh.y, ul.y, dy);
        pair_add(uh.z, ul.z, dz);
        s.lo[v] = make_float4(ul.x, ul.y, ul.z, 0.f);
    } else {
        uh.x += dx;
        uh.y += dy;
        uh.z += dz;
    }
    s.hi[v] = make_float4(uh.x, uh.y, uh.z, 0.f);
}

}  // namespace el
}  // namespace pbng
