// Equilibrium adjoint for sm_103a: H lambda = dL/du by coloured block
// Gauss-Seidel with the true Hessian applied matrix-free, then the
// parameter and boundary sensitivities (see pbng_adjoint in include/pbng.h).
//
// The true energy-density Hessian of the corotated model (Eq. cor, the
// tensor of Eq. hess) acting on a direction dF is
//   dP = 2 mu (dF - dR) + lambda (C : dF) C + lambda (J - 1) dC,
// with C = cof F, dC its (bilinear) variation, and dR = R [w]x where
// (tr S I - S) w = axial(R^T dF - dF^T R), S = R^T F (differentiating
// F = R S with S symmetric).  For vertex i, (H lambda)_i = sum_e V_e dP(dF_e) g_i
// with dF_e = sum_j lambda_j g_j^T, plus the weak terms.
//
// Vertex kernels use the ring layout of pbng_ring.cu (one warp per 32-slot
// item, W lanes per vertex, 1-ring values exchanged by shuffles) with direct
// loads; the block Gauss-Seidel pass also runs pipelined like the colour
// pass (adjoint_ring_sweep_kernel).  The gradient kernel runs one thread per
// tetrahedron.
#include "pbng_async.cuh"
#include "pbng_element.cuh"
#include "pbng_internal.h"

namespace pbng {
namespace {

using el::f3;
using el::kFull;

struct ElemState {
    float H[9];    // F - I
    float C[9];    // cof F
    float Jm1;     // det F - 1
    float RmI[9];  // R - I (corotated only)
    float n2;      // |F|^2
};

// F, its cofactor, J - 1 and the rotation, all from the displacement
// differences dk = u_jk - u_i and the gradients of the other three vertices.
template <int MODEL>
__device__ __forceinline__ void elem_state(float3 d1, float3 d2, float3 d3, float3 g1, float3 g2, float3 g3,
                                           ElemState& E) {
    const float a1[3] = {d1.x, d1.y, d1.z}, a2[3] = {d2.x, d2.y, d2.z}, a3[3] = {d3.x, d3.y, d3.z};
    const float b1[3] = {g1.x, g1.y, g1.z}, b2[3] = {g2.x, g2.y, g2.z}, b3[3] = {g3.x, g3.y, g3.z};
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) E.H[3 * p + q] = a1[p] * b1[q] + a2[p] * b2[q] + a3[p] * b3[q];
    const float* H = E.H;
    const float F0 = 1.0f + H[0], F4 = 1.0f + H[4], F8 = 1.0f + H[8];
    const float F1 = H[1], F2 = H[2], F3 = H[3], F5 = H[5], F6 = H[6], F7 = H[7];
    E.C[0] = F4 * F8 - F5 * F7;
    E.C[1] = F5 * F6 - F3 * F8;
    E.C[2] = F3 * F7 - F4 * F6;
    E.C[3] = F7 * F2 - F8 * F1;
    E.C[4] = F8 * F0 - F6 * F2;
    E.C[5] = F6 * F1 - F7 * F0;
    E.C[6] = F1 * F5 - F2 * F4;
    E.C[7] = F2 * F3 - F0 * F5;
    E.C[8] = F0 * F4 - F1 * F3;
    E.Jm1 = (H[0] + H[4] + H[8]) +
            (H[0] * H[4] - H[1] * H[3] + H[0] * H[8] - H[2] * H[6] + H[4] * H[8] - H[5] * H[7]) +
            el::det3(H[0], H[1], H[2], H[3], H[4], H[5], H[6], H[7], H[8]);
    const float Fm[9] = {F0, F1, F2, F3, F4, F5, F6, F7, F8};
    float n2 = 0.f, c2 = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        n2 += Fm[k] * Fm[k];
        c2 += E.C[k] * E.C[k];
    }
    E.n2 = n2;
    if (MODEL == el::kCorotated) el::rotation_minus_identity(H, n2, c2, 1.0f + E.Jm1, E.RmI);
}

// V dC: the bilinear variation of the cofactor, row i of C being the cross
// product of rows i+1 and i+2 of F.
__device__ __forceinline__ void cof_variation(const float* F, const float* dF, float* dC) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int p = 3 * ((i + 1) % 3), q = 3 * ((i + 2) % 3);
        dC[3 * i] = (dF[p + 1] * F[q + 2] - dF[p + 2] * F[q + 1]) + (F[p + 1] * dF[q + 2] - F[p + 2] * dF[q + 1]);
        dC[3 * i + 1] = (dF[p + 2] * F[q] - dF[p] * F[q + 2]) + (F[p + 2] * dF[q] - F[p] * dF[q + 2]);
        dC[3 * i + 2] = (dF[p] * F[q + 1] - dF[p + 1] * F[q]) + (F[p] * dF[q + 1] - F[p + 1] * dF[q]);
    }
}

// V P (row-major 3x3) of the model (Section "Constitutive Models"), with
// a = 2 mu V, b = lambda V: corotated a (F - R) + b (J - 1) C; Neo-Hookean
// (a/2) (F - C) + (a/2 + b) (J - 1) C; stable Neo-Hookean (Lame-consistent
// mu' = 4mu/3, lambda' = lambda + 5mu/6) (a/2) (F - C) + (a/6) (I_C - 3) /
// (1 + I_C) F + (b + 5a/12) (J - 1) C.
template <int MODEL>
__device__ __forceinline__ void elem_vp(const ElemState& E, float a, float b, float* VP) {
    if (MODEL == el::kCorotated) {
#pragma unroll
        for (int k = 0; k < 9; ++k) VP[k] = a * (E.H[k] - E.RmI[k]) + b * E.Jm1 * E.C[k];
        return;
    }
    const float kv = MODEL == el::kNeoHookean ? 0.5f * a + b : b + a * (5.0f / 12.0f);
    const float qs = MODEL == el::kNeoHookean ? 0.0f : (a * (1.0f / 6.0f)) * (E.n2 - 3.0f) / (1.0f + E.n2);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float F = E.H[k] + ((k % 4 == 0) ? 1.0f : 0.0f);
        VP[k] = 0.5f * a * (F - E.C[k]) + qs * F + kv * E.Jm1 * E.C[k];
    }
}

// out = V dP(dF) (row-major 3x3), a = 2 mu V, b = lambda V.
//   Neo-Hookean: (a/2) dF + (a/2 + b) (C:dF) C + ((a/2 + b)(J - 1) - a/2) dC
//   stable NH:   (2a/3) I_C/(1 + I_C) dF + (4a/3) (F:dF)/(1 + I_C)^2 F
//                + (b + 5a/12) (C:dF) C + ((b + 5a/12)(J - 1) - a/2) dC
template <int MODEL>
__device__ __forceinline__ void hess_action(const ElemState& E, float a, float b, const float* dF, float* out) {
    if (MODEL != el::kCorotated) {
        float F[9], dC[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) F[k] = E.H[k] + ((k % 4 == 0) ? 1.0f : 0.0f);
        cof_variation(F, dF, dC);
        float CdF = 0.f, FdF = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            CdF += E.C[k] * dF[k];
            FdF += F[k] * dF[k];
        }
        const float lv = MODEL == el::kNeoHookean ? 0.5f * a + b : b + a * (5.0f / 12.0f);
        const float ic = E.n2, q = 1.0f + ic;
        const float sv = MODEL == el::kNeoHookean ? 0.5f * a : (2.0f * a / 3.0f) * ic / q;
        const float tv = MODEL == el::kNeoHookean ? 0.0f : (4.0f * a / 3.0f) * FdF / (q * q);
        const float kv = lv * E.Jm1 - 0.5f * a;
#pragma unroll
        for (int k = 0; k < 9; ++k) out[k] = sv * dF[k] + tv * F[k] + lv * CdF * E.C[k] + kv * dC[k];
        return;
    }
    float R[9], F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float id = (k % 4 == 0) ? 1.0f : 0.0f;
        R[k] = E.RmI[k] + id;
        F[k] = E.H[k] + id;
    }
    float S[9], X[9];  // S = R^T F, X = R^T dF
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            S[3 * i + j] = R[i] * F[j] + R[3 + i] * F[3 + j] + R[6 + i] * F[6 + j];
            X[3 * i + j] = R[i] * dF[j] + R[3 + i] * dF[3 + j] + R[6 + i] * dF[6 + j];
        }
    const float r0 = X[7] - X[5], r1 = X[2] - X[6], r2 = X[3] - X[1];
    const float tr = S[0] + S[4] + S[8];
    const float m00 = tr - S[0], m11 = tr - S[4], m22 = tr - S[8];
    const float m01 = -0.5f * (S[1] + S[3]), m02 = -0.5f * (S[2] + S[6]), m12 = -0.5f * (S[5] + S[7]);
    const float c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
    const float c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
    const float det = m00 * c00 + m01 * c01 + m02 * c02;
    float w0 = 0.f, w1 = 0.f, w2 = 0.f;
    if (fabsf(det) > 1e-30f) {
        const float inv = 1.0f / det;
        w0 = inv * (c00 * r0 + c01 * r1 + c02 * r2);
        w1 = inv * (c01 * r0 + c11 * r1 + c12 * r2);
        w2 = inv * (c02 * r0 + c12 * r1 + c22 * r2);
    }
    // dR = R [w]x
    float dR[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float ri0 = R[3 * i], ri1 = R[3 * i + 1], ri2 = R[3 * i + 2];
        dR[3 * i] = ri1 * w2 - ri2 * w1;
        dR[3 * i + 1] = ri2 * w0 - ri0 * w2;
        dR[3 * i + 2] = ri0 * w1 - ri1 * w0;
    }
    // dC: row i of C is (row i+1) x (row i+2) of F
    float dC[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int p = 3 * ((i + 1) % 3), q = 3 * ((i + 2) % 3);
        dC[3 * i] = (dF[p + 1] * F[q + 2] - dF[p + 2] * F[q + 1]) + (F[p + 1] * dF[q + 2] - F[p + 2] * dF[q + 1]);
        dC[3 * i + 1] = (dF[p + 2] * F[q] - dF[p] * F[q + 2]) + (F[p + 2] * dF[q] - F[p] * dF[q + 2]);
        dC[3 * i + 2] = (dF[p] * F[q + 1] - dF[p + 1] * F[q]) + (F[p] * dF[q + 1] - F[p + 1] * dF[q]);
    }
    float CdF = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) CdF += E.C[k] * dF[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = a * (dF[k] - dR[k]) + b * (CdF * E.C[k] + E.Jm1 * dC[k]);
}

__device__ __forceinline__ float3 mat_g(const float* M, float3 g) {
    return make_float3(M[0] * g.x + M[1] * g.y + M[2] * g.z, M[3] * g.x + M[4] * g.y + M[5] * g.z,
                       M[6] * g.x + M[7] * g.y + M[8] * g.z);
}

// kDiag: 3x3 diagonal blocks of H; kSweep: one block Gauss-Seidel pass;
// kResid: |gv - H lam|^2 per warp; kForce: r = f + f^ext at u into out, the
// SPD modified blocks A_i of Eq. mod_hess into diag, |r|^2 per warp;
// kApply: out = H lam (lam = a direction, zero at clamped vertices),
// lam . H lam per warp.
enum { kDiag = 0, kSweep = 1, kResid = 2, kForce = 3, kApply = 4 };

// Two-sided weak constraints (Section "Weak Constraints") in the true
// Hessian: constraint c adds beta_v beta_j K_c to block (v, j), so
// (H lam)_v gains sum_c beta_v K_c (sum_q b_q lam_q) (lam zero at clamped
// vertices) and the diagonal block sum_c beta_v^2 K_c (the same term as in
// Eq. mod_hess).  h (3) and D (upper triangle, 6, or nullptr) are added to.
__device__ __forceinline__ void weak_hessian(const DeviceMesh& m, const float4* lam, int v, float* h, float* D) {
    if (!m.wc_off) return;
    const int k1 = m.wc_off[v + 1];
    for (int k = m.wc_off[v]; k < k1; ++k) {
        const int2 e = m.wc_list[k];
        const int c = e.x;
        const float beta = __int_as_float(e.y);
        float Cl[3] = {0.f, 0.f, 0.f};
        if (h) {
            for (int q = 0; q < 8; ++q) {
                const int jq = m.wc_v[8 * c + q];
                if (jq < 0) break;
                const float bq = m.wc_b[8 * c + q];
                const float4 l = lam[jq];
                Cl[0] += bq * l.x;
                Cl[1] += bq * l.y;
                Cl[2] += bq * l.z;
            }
        }
        const float* K = m.wc_k + 6 * c;
        if (h) {
            h[0] += beta * (K[0] * Cl[0] + K[1] * Cl[1] + K[2] * Cl[2]);
            h[1] += beta * (K[1] * Cl[0] + K[3] * Cl[1] + K[4] * Cl[2]);
            h[2] += beta * (K[2] * Cl[0] + K[4] * Cl[1] + K[5] * Cl[2]);
        }
        if (D) {
            const float b2 = beta * beta;
#pragma unroll
            for (int t = 0; t < 6; ++t) D[t] += b2 * K[t];
        }
    }
}

template <int W, int MODE, int MODEL>
__device__ __forceinline__ void adj_item(const DeviceMesh& m, const State& u, float4* lam, const float4* gv,
                                         float4* diag, float4* out4, const Item& it, int lane, int32_t* err,
                                         double& rr) {
    const int j = lane / W;
    const bool active = j < it.nv;
    const int v = it.v0 + j;
    const int slot = it.slot0 + lane;
    const float3 z3 = make_float3(0.f, 0.f, 0.f);
    float3 uh = z3, ul = z3, li = z3, du = z3, dl = z3;
    if (active) {
        uh = f3(u.hi[v]);
        ul = f3(u.lo[v]);
        if (MODE != kForce) li = f3(lam[v]);
        const int id = m.ring[slot >> 5].id[slot & 31];
        du = el::pair_diff<true>(u.hi[id], u.lo[id], uh, ul);
        if (MODE != kDiag && MODE != kForce) {
            const float3 lj = f3(lam[id]);
            dl = make_float3(lj.x - li.x, lj.y - li.y, lj.z - li.z);
        }
    }
    const RingBlock& rbk = m.ring[slot >> 5];
    const float4 ra = rbk.ra[slot & 31], rb = rbk.rb[slot & 31], rc = rbk.rc[slot & 31];
    const int loc = __float_as_int(rc.w);
    const int base = lane & ~(W - 1);
    const int s[3] = {base + (loc & 255), base + ((loc >> 8) & 255), base + ((loc >> 16) & 255)};
    float3 d[3], e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d[k] = make_float3(__shfl_sync(kFull, du.x, s[k]), __shfl_sync(kFull, du.y, s[k]), __shfl_sync(kFull, du.z, s[k]));
        e[k] = make_float3(__shfl_sync(kFull, dl.x, s[k]), __shfl_sync(kFull, dl.y, s[k]), __shfl_sync(kFull, dl.z, s[k]));
    }
    const float3 g1 = f3(ra), g2 = f3(rb), g3 = f3(rc);
    const float3 gi = make_float3(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
    ElemState E;
    elem_state<MODEL>(d[0], d[1], d[2], g1, g2, g3, E);
    float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float out[9];
    if (MODE == kForce) {
        // -V P g_i (Eq. cor) and V (2 mu |g_i|^2 I + lambda w w^T), w = cof(F) g_i
        const float3 w = mat_g(E.C, gi);
        const float a = ra.w, b = rb.w;
        float VP[9];
        elem_vp<MODEL>(E, a, b, VP);
        const float3 fr = mat_g(VP, gi);
        acc[0] = -fr.x;
        acc[1] = -fr.y;
        acc[2] = -fr.z;
        const float ag = a * (gi.x * gi.x + gi.y * gi.y + gi.z * gi.z);
        acc[3] = ag + b * w.x * w.x;
        acc[4] = b * w.x * w.y;
        acc[5] = b * w.x * w.z;
        acc[6] = ag + b * w.y * w.y;
        acc[7] = b * w.y * w.z;
        acc[8] = ag + b * w.z * w.z;
    } else if (MODE == kDiag) {
        const float gg[3] = {gi.x, gi.y, gi.z};
        float col[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float dF[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            dF[3 * c] = gg[0];
            dF[3 * c + 1] = gg[1];
            dF[3 * c + 2] = gg[2];
            hess_action<MODEL>(E, ra.w, rb.w, dF, out);
            const float3 h = mat_g(out, gi);
            col[c][0] = h.x;
            col[c][1] = h.y;
            col[c][2] = h.z;
        }
        acc[0] = col[0][0];
        acc[1] = col[1][0];
        acc[2] = col[2][0];
        acc[3] = col[1][1];
        acc[4] = col[2][1];
        acc[5] = col[2][2];
    } else {
        const float dF[9] = {e[0].x * g1.x + e[1].x * g2.x + e[2].x * g3.x, e[0].x * g1.y + e[1].x * g2.y + e[2].x * g3.y,
                             e[0].x * g1.z + e[1].x * g2.z + e[2].x * g3.z, e[0].y * g1.x + e[1].y * g2.x + e[2].y * g3.x,
                             e[0].y * g1.y + e[1].y * g2.y + e[2].y * g3.y, e[0].y * g1.z + e[1].y * g2.z + e[2].y * g3.z,
                             e[0].z * g1.x + e[1].z * g2.x + e[2].z * g3.x, e[0].z * g1.y + e[1].z * g2.y + e[2].z * g3.y,
                             e[0].z * g1.z + e[1].z * g2.z + e[2].z * g3.z};
        hess_action<MODEL>(E, ra.w, rb.w, dF, out);
        const float3 h = mat_g(out, gi);
        acc[0] = h.x;
        acc[1] = h.y;
        acc[2] = h.z;
    }
    constexpr int NA = (MODE == kForce) ? 9 : ((MODE == kDiag) ? 6 : 3);
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = el::group_sum<W>(acc[k]);
    if (!active || (lane & (W - 1)) != 0) return;
    if (MODE == kForce) {
        float r[3] = {acc[0], acc[1], acc[2]};
        float A[6] = {acc[3], acc[4], acc[5], acc[6], acc[7], acc[8]};
        el::vertex_terms<true, true>(m, m.aux0[v], m.aux1[v], uh, ul, r, A);
        el::weak_terms<true, true>(m, u, v, r, A);
        out4[v] = make_float4(r[0], r[1], r[2], 0.f);
        diag[2 * v] = make_float4(A[0], A[1], A[2], A[3]);
        diag[2 * v + 1] = make_float4(A[4], A[5], 0.f, 0.f);
        rr += (double)r[0] * r[0] + (double)r[1] * r[1] + (double)r[2] * r[2];
        return;
    }
    // weak terms: springs K I, active plane contact k n n^T
    const float4 x0 = m.aux0[v], x1 = m.aux1[v];
    const float K = x0.w;
    bool contact = false;
    if (m.k_contact > 0.0f) {
        const float sd = x1.w + (m.pn_x * (uh.x + ul.x) + m.pn_y * (uh.y + ul.y) + m.pn_z * (uh.z + ul.z));
        contact = sd < 0.0f;
    }
    const float kc = contact ? m.k_contact : 0.0f;
    const float n[3] = {m.pn_x, m.pn_y, m.pn_z};
    if (MODE == kDiag) {
        acc[0] += K + kc * n[0] * n[0];
        acc[1] += kc * n[0] * n[1];
        acc[2] += kc * n[0] * n[2];
        acc[3] += K + kc * n[1] * n[1];
        acc[4] += kc * n[1] * n[2];
        acc[5] += K + kc * n[2] * n[2];
        weak_hessian(m, lam, v, nullptr, acc);
        diag[2 * v] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        diag[2 * v + 1] = make_float4(acc[4], acc[5], 0.f, 0.f);
        return;
    }
    const float nl = kc * (n[0] * li.x + n[1] * li.y + n[2] * li.z);
    weak_hessian(m, lam, v, acc, nullptr);
    if (MODE == kApply) {
        const float h0 = acc[0] + K * li.x + nl * n[0], h1 = acc[1] + K * li.y + nl * n[1],
                    h2 = acc[2] + K * li.z + nl * n[2];
        out4[v] = make_float4(h0, h1, h2, 0.f);
        rr += (double)li.x * h0 + (double)li.y * h1 + (double)li.z * h2;
        return;
    }
    const float4 gvv = gv[v];
    const float r0 = gvv.x - (acc[0] + K * li.x + nl * n[0]);
    const float r1 = gvv.y - (acc[1] + K * li.y + nl * n[1]);
    const float r2 = gvv.z - (acc[2] + K * li.z + nl * n[2]);
    if (MODE == kResid) {
        rr += (double)r0 * r0 + (double)r1 * r1 + (double)r2 * r2;
        return;
    }
    const float4 D0 = diag[2 * v], D1 = diag[2 * v + 1];
    const float A[6] = {D0.x, D0.y, D0.z, D0.w, D1.x, D1.y};
    const float c00 = A[3] * A[5] - A[4] * A[4], c01 = A[2] * A[4] - A[1] * A[5], c02 = A[1] * A[4] - A[2] * A[3];
    const float c11 = A[0] * A[5] - A[2] * A[2], c12 = A[1] * A[2] - A[0] * A[4], c22 = A[0] * A[3] - A[1] * A[1];
    const float det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(det > 0.0f) || !(det < 3.0e38f)) {
        atomicOr(err, kErrNonSPD);
        return;
    }
    const float inv = 1.0f / det;
    lam[v] = make_float4(li.x + inv * (c00 * r0 + c01 * r1 + c02 * r2), li.y + inv * (c01 * r0 + c11 * r1 + c12 * r2),
                         li.z + inv * (c02 * r0 + c12 * r1 + c22 * r2), 0.f);
}

template <int MODE, int MODEL>
__global__ void __launch_bounds__(kBlock, 3) adjoint_vertex_kernel(const DeviceMesh m, State u, float4* lam,
                                                                const float4* gv, float4* diag, float4* out4,
                                                                const Item* __restrict__ items, int nitems,
                                                                int32_t* err, double* partial) {
    const int lane = threadIdx.x & 31;
    const int gw = (int)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
    double rr = 0.0;
    if (gw < nitems) {
        const Item it = items[gw];
        switch (it.w) {
            case 4: adj_item<4, MODE, MODEL>(m, u, lam, gv, diag, out4, it, lane, err, rr); break;
            case 8: adj_item<8, MODE, MODEL>(m, u, lam, gv, diag, out4, it, lane, err, rr); break;
            case 16: adj_item<16, MODE, MODEL>(m, u, lam, gv, diag, out4, it, lane, err, rr); break;
            default: adj_item<32, MODE, MODEL>(m, u, lam, gv, diag, out4, it, lane, err, rr); break;
        }
    }
    if (MODE == kResid || MODE == kForce || MODE == kApply) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) rr += __shfl_xor_sync(kFull, rr, off);
        if (lane == 0) partial[gw] = rr;
    }
}

// One thread per tet: dL/dlog E_e = -sum_{j free} lambda_j . (V P g_j), and,
// for tets touching clamped vertices, (H_DF lambda)_d += V dP(dF) g_d with
// dF = sum_j lambda_j g_j^T (lambda = 0 at clamped vertices).
template <int MODEL>
__global__ void adjoint_tet_kernel(int ne, int nfree, const int4* __restrict__ tv, const float4* __restrict__ tb,
                                   State u, const float4* __restrict__ lam, float* dLdlogE, float* hdl) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int4 t = tv[e];
    const int ids[4] = {t.x, t.y, t.z, t.w};
    const float4 B0 = tb[3 * e], B1 = tb[3 * e + 1], B2 = tb[3 * e + 2];
    const float a = B0.w, b = B1.w;
    float3 g[4];
    g[1] = f3(B0);
    g[2] = f3(B1);
    g[3] = f3(B2);
    g[0] = make_float3(-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z));
    const float3 u0h = f3(u.hi[ids[0]]), u0l = f3(u.lo[ids[0]]);
    float3 d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = el::pair_diff<true>(u.hi[ids[k + 1]], u.lo[ids[k + 1]], u0h, u0l);
    ElemState E;
    elem_state<MODEL>(d[0], d[1], d[2], g[1], g[2], g[3], E);
    float VP[9];
    elem_vp<MODEL>(E, a, b, VP);
    float3 L[4];
    float grad = 0.f;
    bool touches = false;
#pragma unroll
    for (int jv = 0; jv < 4; ++jv) {
        if (ids[jv] < nfree) {
            L[jv] = f3(lam[ids[jv]]);
            const float3 pg = mat_g(VP, g[jv]);
            grad -= L[jv].x * pg.x + L[jv].y * pg.y + L[jv].z * pg.z;
        } else {
            L[jv] = make_float3(0.f, 0.f, 0.f);
            touches = true;
        }
    }
    dLdlogE[e] = grad;
    if (!touches) return;
    float dF[9];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const float lp[4] = {p == 0 ? L[0].x : (p == 1 ? L[0].y : L[0].z), p == 0 ? L[1].x : (p == 1 ? L[1].y : L[1].z),
                             p == 0 ? L[2].x : (p == 1 ? L[2].y : L[2].z), p == 0 ? L[3].x : (p == 1 ? L[3].y : L[3].z)};
        dF[3 * p] = lp[0] * g[0].x + lp[1] * g[1].x + lp[2] * g[2].x + lp[3] * g[3].x;
        dF[3 * p + 1] = lp[0] * g[0].y + lp[1] * g[1].y + lp[2] * g[2].y + lp[3] * g[3].y;
        dF[3 * p + 2] = lp[0] * g[0].z + lp[1] * g[1].z + lp[2] * g[2].z + lp[3] * g[3].z;
    }
    float out[9];
    hess_action<MODEL>(E, a, b, dF, out);
#pragma unroll
    for (int jv = 0; jv < 4; ++jv)
        if (ids[jv] >= nfree) {
            const float3 h = mat_g(out, g[jv]);
            atomicAdd(hdl + 4 * ids[jv], h.x);
            atomicAdd(hdl + 4 * ids[jv] + 1, h.y);
            atomicAdd(hdl + 4 * ids[jv] + 2, h.z);
        }
}

// H_DF lam of the two-sided weak constraints: each constraint c with a
// clamped vertex D adds b_D K_c (sum_q b_q lam_q) to hdl[D] (lam zero at
// clamped vertices); one thread per constraint.
__global__ void adjoint_weak_clamped_kernel(int nwc, int nfree, const DeviceMesh m, const float4* __restrict__ lam,
                                            float* hdl) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nwc) return;
    bool any = false;
    float Cl[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < 8; ++q) {
        const int jq = m.wc_v[8 * c + q];
        if (jq < 0) break;
        any = any || jq >= nfree;
        const float bq = m.wc_b[8 * c + q];
        const float4 l = lam[jq];
        Cl[0] += bq * l.x;
        Cl[1] += bq * l.y;
        Cl[2] += bq * l.z;
    }
    if (!any) return;
    const float* K = m.wc_k + 6 * c;
    const float KC[3] = {K[0] * Cl[0] + K[1] * Cl[1] + K[2] * Cl[2], K[1] * Cl[0] + K[3] * Cl[1] + K[4] * Cl[2],
                         K[2] * Cl[0] + K[4] * Cl[1] + K[5] * Cl[2]};
    for (int q = 0; q < 8; ++q) {
        const int jq = m.wc_v[8 * c + q];
        if (jq < 0) break;
        if (jq < nfree) continue;
        const float bq = m.wc_b[8 * c + q];
        atomicAdd(hdl + 4 * jq, bq * KC[0]);
        atomicAdd(hdl + 4 * jq + 1, bq * KC[1]);
        atomicAdd(hdl + 4 * jq + 2, bq * KC[2]);
    }
}

// Refined adjoint: the shifted states u +- eps lam for the central difference
// of the float-float force.
__global__ void adjoint_shift_kernel(int nv, State u, const float4* __restrict__ lh, const float4* __restrict__ ll,
                                     float eps, State up, State um) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const float4 uh = u.hi[v], ul = u.lo[v], a = lh[v], b = ll[v];
    const float uhv[3] = {uh.x, uh.y, uh.z}, ulv[3] = {ul.x, ul.y, ul.z};
    const float av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z};
    float ph[3], pl[3], mh[3], ml[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const ff::F2 x = ff::mk(uhv[k], ulv[k]);
        const ff::F2 d = ff::mul(ff::add(ff::mk(av[k]), bv[k]), eps);
        const ff::F2 p = ff::add(x, d), q = ff::sub(x, d);
        ph[k] = p.h;
        pl[k] = p.l;
        mh[k] = q.h;
        ml[k] = q.l;
    }
    up.hi[v] = make_float4(ph[0], ph[1], ph[2], 0.f);
    up.lo[v] = make_float4(pl[0], pl[1], pl[2], 0.f);
    um.hi[v] = make_float4(mh[0], mh[1], mh[2], 0.f);
    um.lo[v] = make_float4(ml[0], ml[1], ml[2], 0.f);
}

constexpr int kVecBlock = 256;

__global__ void __launch_bounds__(kVecBlock) adjoint_refine_rhs_kernel(int n, const float4* __restrict__ gv,
                                                                      const float4* __restrict__ ph,
                                                                      const float4* __restrict__ pl,
                                                                      const float4* __restrict__ mh,
                                                                      const float4* __restrict__ ml, double inv2eps,
                                                                      float4* rhs, double* partial) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    double q = 0.0;
    if (w < n) {
        const float4 g = gv[w], a = ph[w], b = pl[w], c = mh[w], d = ml[w];
        const double r0 = (double)g.x + (((double)a.x + b.x) - ((double)c.x + d.x)) * inv2eps;
        const double r1 = (double)g.y + (((double)a.y + b.y) - ((double)c.y + d.y)) * inv2eps;
        const double r2 = (double)g.z + (((double)a.z + b.z) - ((double)c.z + d.z)) * inv2eps;
        rhs[w] = make_float4((float)r0, (float)r1, (float)r2, 0.f);
        q = r0 * r0 + r1 * r1 + r2 * r2;
    }
    __shared__ double sh[kVecBlock];
    sh[threadIdx.x] = q;
    __syncthreads();
    for (int k = kVecBlock / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void adjoint_accumulate_kernel(int n, const float4* __restrict__ d, float4* lh, float4* ll, float* maxabs) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n) return;
    const float4 a = lh[w], b = ll[w], e = d[w];
    const float av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z}, ev[3] = {e.x, e.y, e.z};
    float h[3], l[3], mx = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const ff::F2 s = ff::add(ff::mk(av[k], bv[k]), ev[k]);
        h[k] = s.h;
        l[k] = s.l;
        mx = fmaxf(mx, fabsf(s.h));
    }
    lh[w] = make_float4(h[0], h[1], h[2], 0.f);
    ll[w] = make_float4(l[0], l[1], l[2], 0.f);
    atomicMax(reinterpret_cast<int*>(maxabs), __float_as_int(mx));  // non-negative floats order as ints
}

// Conjugate gradients on the adjoint system (PBNG_ACCEL_CG), over the n
// free rows: one FP64 partial per kVecBlock-thread block.
__device__ __forceinline__ void vec_block_partial(double q, double* partial) {
    __shared__ double sh[kVecBlock];
    sh[threadIdx.x] = q;
    __syncthreads();
    for (int k = kVecBlock / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// x += a p, r -= a q with a = sc[0] / sc[1] (r . z over p . H p, on the
// device); partial: |r|^2.  A non-positive or non-finite p . H p (H not
// positive definite) sets *flag and leaves x and r as they are.
__global__ void __launch_bounds__(kVecBlock) acg_step_kernel(int n, const double* sc, int32_t* flag,
                                                             const float4* __restrict__ p,
                                                             const float4* __restrict__ q, float4* x, float4* r,
                                                             double* partial) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const double pq = sc[1];
    const bool ok = pq > 0.0 && pq < 1e300 && !*flag;
    if (!ok && w == 0) *flag = 1;
    const float a = ok ? (float)(sc[0] / pq) : 0.0f;
    double s = 0.0;
    if (w < n) {
        const float4 rw = r[w];
        float4 rn = rw;
        if (ok) {
            const float4 pw = p[w], qw = q[w], xw = x[w];
            x[w] = make_float4(xw.x + a * pw.x, xw.y + a * pw.y, xw.z + a * pw.z, 0.f);
            rn = make_float4(rw.x - a * qw.x, rw.y - a * qw.y, rw.z - a * qw.z, 0.f);
            r[w] = rn;
        }
        s = (double)rn.x * rn.x + (double)rn.y * rn.y + (double)rn.z * rn.z;
    }
    vec_block_partial(s, partial);
}

// partial: r . z
__global__ void __launch_bounds__(kVecBlock) acg_dot_kernel(int n, const float4* __restrict__ r,
                                                            const float4* __restrict__ z, double* partial) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (w < n) {
        const float4 a = r[w], b = z[w];
        s = (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z;
    }
    vec_block_partial(s, partial);
}

// gvec[w] = dL/du of internal free vertex w (caller layout in).
__global__ void gather_rhs_kernel(int nfree, const int32_t* perm, const float* dLdu, float4* gv) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nfree) return;
    const int o = perm[w];
    gv[w] = make_float4(dLdu[3 * o], dLdu[3 * o + 1], dLdu[3 * o + 2], 0.f);
}

// dL/dx_D[q] = dL/du(clamped vertex) - (H_DF lambda)(that vertex).
__global__ void clamped_grad_kernel(int nd, const int32_t* dq_internal, const int32_t* dq_caller,
                                    const float* dLdu, const float* hdl, float* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nd) return;
    const int w = dq_internal[q], o = dq_caller[q];
    out[3 * q] = dLdu[3 * o] - hdl[4 * w];
    out[3 * q + 1] = dLdu[3 * o + 1] - hdl[4 * w + 1];
    out[3 * q + 2] = dLdu[3 * o + 2] - hdl[4 * w + 2];
}

inline int nblocks(int n, int b) { return (n + b - 1) / b; }

// ---- block Gauss-Seidel pass, pipelined -----------------------------------
// The kSweep pass of adj_item with the colour pass's pipeline: persistent
// warps, each item's record block by a TMA bulk copy two items ahead; the
// 1-ring displacement pairs and multipliers, and the own vertices'
// displacement pair, multiplier, right-hand side, diagonal block and aux
// records, by cp.async one item ahead.  The multipliers a pass gathers belong
// to other colours, and an item's own vertices are written only by its warp
// after they were read, so the result is the direct-load pass's.
using namespace async;

constexpr int kAdjWarps = 6;  // per CTA
constexpr int kAdjCtasPerSm = 3;
constexpr int kAdjRecStages = 3;
constexpr int kAdjGatStages = 2;
constexpr int kAdjItemVerts = kRingLanes / 4;

struct __align__(16) AdjGat {
    float4 nh[kRingLanes];     // 1-ring displacement hi
    float4 nl[kRingLanes];     // 1-ring displacement lo
    float4 nlam[kRingLanes];   // 1-ring multiplier
    float4 oh[kAdjItemVerts];  // own displacement hi, lo, multiplier, dL/du
    float4 ol[kAdjItemVerts];
    float4 olam[kAdjItemVerts];
    float4 ogv[kAdjItemVerts];
    float4 od0[kAdjItemVerts];  // own diagonal block (two float4)
    float4 od1[kAdjItemVerts];
    float4 oa0[kAdjItemVerts];  // own aux records
    float4 oa1[kAdjItemVerts];
};

struct __align__(16) AdjWarpSmem {
    RingBlock rec[kAdjRecStages];
    AdjGat gat[kAdjGatStages];
    Item desc[kAdjRecStages];
    unsigned long long bar[kAdjRecStages];
};

static_assert(kAdjCtasPerSm * (kAdjWarps * sizeof(AdjWarpSmem) + 1024) <= 228 * 1024,
              "the adjoint pass's per-warp stages exceed an SM's shared memory");
static_assert(sizeof(RingBlock) % 16 == 0, "bulk copies move multiples of 16 bytes");

__device__ __forceinline__ void adj_issue_records(const DeviceMesh& m, Item it, AdjWarpSmem& S, int r) {
    S.desc[r] = it;
    mbar_arrive_expect_tx(S.bar + r, (uint32_t)sizeof(RingBlock));
    bulk_g2s(&S.rec[r], m.ring + (it.slot0 >> 5), (uint32_t)sizeof(RingBlock), S.bar + r);
}

// APPLY: the Hessian action needs neither the right-hand side nor the
// diagonal block.
template <bool APPLY>
__device__ __forceinline__ void adj_issue_gathers(const DeviceMesh& m, const State& u, const float4* lam,
                                                  const float4* gv, const float4* diag, AdjWarpSmem& S, int r,
                                                  int g, int lane) {
    const Item it = S.desc[r];
    AdjGat& G = S.gat[g];
    const int id = S.rec[r].id[lane];
    cp_async16(G.nh + lane, u.hi + id);
    cp_async16(G.nl + lane, u.lo + id);
    cp_async16(G.nlam + lane, lam + id);
    if (lane < it.nv) {
        const int v = it.v0 + lane;
        cp_async16(G.oh + lane, u.hi + v);
        cp_async16(G.ol + lane, u.lo + v);
        cp_async16(G.olam + lane, lam + v);
        if (!APPLY) {
            cp_async16(G.ogv + lane, gv + v);
            cp_async16(G.od0 + lane, diag + 2 * v);
            cp_async16(G.od1 + lane, diag + 2 * v + 1);
        }
        cp_async16(G.oa0 + lane, m.aux0 + v);
        cp_async16(G.oa1 + lane, m.aux1 + v);
    }
}

// APPLY: instead of the Gauss-Seidel update, hout[v] = (H lam)_v and
// rr += lam_v . (H lam)_v.
template <int W>
__device__ __forceinline__ void adj_group_sums(float* acc) {
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] = el::group_sum<W>(acc[k]);
}

// The lane width W = it.w is a run-time value everywhere but in the W-lane
// sums, so the kernel holds one copy of the element state and Hessian action.
template <int MODEL, bool APPLY>
__device__ __forceinline__ void adj_ring_item(const DeviceMesh& m, float4* lam, const AdjWarpSmem& S, int r, int g,
                                              int lane, int32_t* err, float4* hout, double& rr) {
    const Item it = S.desc[r];
    const RingBlock& R = S.rec[r];
    const AdjGat& G = S.gat[g];
    const int W = it.w;
    const int j = lane >> (__ffs(W) - 1);
    const bool active = j < it.nv;
    const int v = it.v0 + j;
    const float3 z3 = make_float3(0.f, 0.f, 0.f);
    float3 uh = z3, ul = z3, li = z3, du = z3, dl = z3;
    if (active) {
        uh = f3(G.oh[j]);
        ul = f3(G.ol[j]);
        li = f3(G.olam[j]);
        du = el::pair_diff<true>(G.nh[lane], G.nl[lane], uh, ul);
        const float3 lj = f3(G.nlam[lane]);
        dl = make_float3(lj.x - li.x, lj.y - li.y, lj.z - li.z);
    }
    const float4 ra = R.ra[lane], rb = R.rb[lane], rc = R.rc[lane];
    const int loc = __float_as_int(rc.w);
    const int base = lane & ~(W - 1);
    const int sl[3] = {base + (loc & 255), base + ((loc >> 8) & 255), base + ((loc >> 16) & 255)};
    float3 d[3], e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d[k] = make_float3(__shfl_sync(kFull, du.x, sl[k]), __shfl_sync(kFull, du.y, sl[k]),
                           __shfl_sync(kFull, du.z, sl[k]));
        e[k] = make_float3(__shfl_sync(kFull, dl.x, sl[k]), __shfl_sync(kFull, dl.y, sl[k]),
                           __shfl_sync(kFull, dl.z, sl[k]));
    }
    const float3 g1 = f3(ra), g2 = f3(rb), g3 = f3(rc);
    const float3 gi = make_float3(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
    ElemState E;
    elem_state<MODEL>(d[0], d[1], d[2], g1, g2, g3, E);
    const float dF[9] = {e[0].x * g1.x + e[1].x * g2.x + e[2].x * g3.x, e[0].x * g1.y + e[1].x * g2.y + e[2].x * g3.y,
                         e[0].x * g1.z + e[1].x * g2.z + e[2].x * g3.z, e[0].y * g1.x + e[1].y * g2.x + e[2].y * g3.x,
                         e[0].y * g1.y + e[1].y * g2.y + e[2].y * g3.y, e[0].y * g1.z + e[1].y * g2.z + e[2].y * g3.z,
                         e[0].z * g1.x + e[1].z * g2.x + e[2].z * g3.x, e[0].z * g1.y + e[1].z * g2.y + e[2].z * g3.y,
                         e[0].z * g1.z + e[1].z * g2.z + e[2].z * g3.z};
    float out[9];
    hess_action<MODEL>(E, ra.w, rb.w, dF, out);
    const float3 h = mat_g(out, gi);
    float acc[3] = {h.x, h.y, h.z};
    switch (W) {  // warp-uniform
        case 4: adj_group_sums<4>(acc); break;
        case 8: adj_group_sums<8>(acc); break;
        case 16: adj_group_sums<16>(acc); break;
        default: adj_group_sums<32>(acc); break;
    }
    if (!active || (lane & (W - 1)) != 0) return;
    // weak terms: springs K I, active plane contact k n n^T
    const float4 x0 = G.oa0[j], x1 = G.oa1[j];
    const float K = x0.w;
    bool contact = false;
    if (m.k_contact > 0.0f) {
        const float sd = x1.w + (m.pn_x * (uh.x + ul.x) + m.pn_y * (uh.y + ul.y) + m.pn_z * (uh.z + ul.z));
        contact = sd < 0.0f;
    }
    const float kc = contact ? m.k_contact : 0.0f;
    const float n[3] = {m.pn_x, m.pn_y, m.pn_z};
    const float nl = kc * (n[0] * li.x + n[1] * li.y + n[2] * li.z);
    // the multipliers of a constraint's other vertices belong to other
    // colours (a constraint is an element of the colouring)
    weak_hessian(m, lam, v, acc, nullptr);
    if constexpr (APPLY) {
        const float h0 = acc[0] + K * li.x + nl * n[0], h1 = acc[1] + K * li.y + nl * n[1],
                    h2 = acc[2] + K * li.z + nl * n[2];
        hout[v] = make_float4(h0, h1, h2, 0.f);
        rr += (double)li.x * h0 + (double)li.y * h1 + (double)li.z * h2;
        return;
    }
    const float4 gvv = G.ogv[j];
    const float r0 = gvv.x - (acc[0] + K * li.x + nl * n[0]);
    const float r1 = gvv.y - (acc[1] + K * li.y + nl * n[1]);
    const float r2 = gvv.z - (acc[2] + K * li.z + nl * n[2]);
    const float4 D0 = G.od0[j], D1 = G.od1[j];
    const float A[6] = {D0.x, D0.y, D0.z, D0.w, D1.x, D1.y};
    const float c00 = A[3] * A[5] - A[4] * A[4], c01 = A[2] * A[4] - A[1] * A[5], c02 = A[1] * A[4] - A[2] * A[3];
    const float c11 = A[0] * A[5] - A[2] * A[2], c12 = A[1] * A[2] - A[0] * A[4], c22 = A[0] * A[3] - A[1] * A[1];
    const float det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(det > 0.0f) || !(det < 3.0e38f)) {
        atomicOr(err, kErrNonSPD);
        return;
    }
    const float inv = 1.0f / det;
    lam[v] = make_float4(li.x + inv * (c00 * r0 + c01 * r1 + c02 * r2), li.y + inv * (c01 * r0 + c11 * r1 + c12 * r2),
                         li.z + inv * (c02 * r0 + c12 * r1 + c22 * r2), 0.f);
}

// Warp gw takes items gw, gw + nw, ... of one colour.  Every wait is bounded:
// on a timeout the warp records it, lets its copies land (bounded) and
// returns.
// APPLY: the Hessian action of lam over the given items (any colours; lam
// is only read), with one FP64 partial of lam . H lam per warp of the grid.
template <int MODEL, bool APPLY>
__global__ void __launch_bounds__(kAdjWarps * 32, kAdjCtasPerSm)
    adjoint_ring_sweep_kernel(const DeviceMesh m, State u, float4* lam, const float4* __restrict__ gv,
                              const float4* __restrict__ diag, const Item* __restrict__ items, int nitems,
                              int32_t* err, float4* out, double* partial) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    AdjWarpSmem& S = reinterpret_cast<AdjWarpSmem*>(smem)[warp];
    const int gw = (int)blockIdx.x * kAdjWarps + warp, nw = (int)gridDim.x * kAdjWarps;
    const int n = gw < nitems ? (nitems - gw + nw - 1) / nw : 0;
    const int first = gw, stride = nw;
    int issued = 0, waited = 0;  // items whose records were requested / awaited
    bool ok = true;
    double rr = 0.0;
    Item next{};                 // lane 0: next item to request, loaded one item early
    if (n > 0) {
        if (lane == 0) {
            for (int i = 0; i < kAdjRecStages; ++i) mbar_init(S.bar + i, 1);
            fence_mbar_init();
            for (int i = 0; i < kAdjRecStages - 1 && i < n; ++i) adj_issue_records(m, items[first + i * stride], S, i);
            if (n > kAdjRecStages - 1) next = items[first + (kAdjRecStages - 1) * stride];
        }
        issued = n < kAdjRecStages - 1 ? n : kAdjRecStages - 1;
        __syncwarp();
        ok = mbar_wait(S.bar + 0, 0);
        waited = ok ? 1 : 0;  // a stage whose wait gave up is drained again on abort
        if (__any_sync(kFull, !ok)) goto abort;
        adj_issue_gathers<APPLY>(m, u, lam, gv, diag, S, 0, 0, lane);
        cp_async_commit();
        for (int k = 0; k < n; ++k) {
            // Record stage (k + 2) % 3 and gather stage (k + 1) % 2 were last
            // read by item k - 1, finished before the previous __syncwarp.
            if (k + kAdjRecStages - 1 < n) {
                if (lane == 0) {
                    fence_proxy_async();
                    adj_issue_records(m, next, S, (k + kAdjRecStages - 1) % kAdjRecStages);
                    if (k + kAdjRecStages < n) next = items[first + (k + kAdjRecStages) * stride];
                }
                issued = k + kAdjRecStages;
            }
            ok = true;
            if (k + 1 < n) {
                ok = mbar_wait(S.bar + (k + 1) % kAdjRecStages, ((k + 1) / kAdjRecStages) & 1);
                waited = ok ? k + 2 : k + 1;
                if (ok)
                    adj_issue_gathers<APPLY>(m, u, lam, gv, diag, S, (k + 1) % kAdjRecStages, (k + 1) % kAdjGatStages,
                                             lane);
            }
            cp_async_commit();
            cp_async_wait<1>();  // this lane's gathers of item k have landed
            if (__any_sync(kFull, !ok)) goto abort;
            __syncwarp();        // ... and the other lanes'
            const int r = k % kAdjRecStages, g = k % kAdjGatStages;
            adj_ring_item<MODEL, APPLY>(m, lam, S, r, g, lane, err, out, rr);
            __syncwarp();
        }
    }
    if (APPLY) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) rr += __shfl_xor_sync(kFull, rr, off);
        if (lane == 0) partial[gw] = rr;
    }
    return;

abort:
    if (lane == 0) {
        atomicOr(err, kErrTimeout);
        for (int k = waited; k < issued; ++k) (void)mbar_wait(S.bar + k % kAdjRecStages, (k / kAdjRecStages) & 1);
        if (APPLY) partial[gw] = 0.0;
    }
    cp_async_wait<0>();
    __syncwarp();
}

int adj_sm_count() {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return 148;
    return nsm;
}


// ---- preconditioned conjugate gradients on H x = r (free vertices) --------
// Scalars live on the device: sc[0] = r.z, sc[1] = p.Hp, sc[2] = new r.z,
// sc[3] = |r|^2.  A direction with p.Hp <= 0 (H not positive definite along
// it) sets *flag and freezes every later update (truncated CG).

// z = A^{-1} r for the SPD 3x3 block A (upper triangle in two float4).
__device__ __forceinline__ float3 block_solve(float4 D0, float4 D1, float3 r) {
    const float A[6] = {D0.x, D0.y, D0.z, D0.w, D1.x, D1.y};
    const float c00 = A[3] * A[5] - A[4] * A[4], c01 = A[2] * A[4] - A[1] * A[5], c02 = A[1] * A[4] - A[2] * A[3];
    const float c11 = A[0] * A[5] - A[2] * A[2], c12 = A[1] * A[2] - A[0] * A[4], c22 = A[0] * A[3] - A[1] * A[1];
    const float det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    const float inv = det > 0.0f ? 1.0f / det : 0.0f;
    return make_float3(inv * (c00 * r.x + c01 * r.y + c02 * r.z), inv * (c01 * r.x + c11 * r.y + c12 * r.z),
                       inv * (c02 * r.x + c12 * r.y + c22 * r.z));
}

// One FP64 partial per block, summed in a fixed order.  Ends with a barrier
// so that a second call in the same kernel cannot overwrite ws while thread 0
// still reads it.
__device__ __forceinline__ void block_partial(double v, double* partial) {
    __shared__ double ws[kBlock / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) t += ws[k];
        partial[blockIdx.x] = t;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBlock) cg_init_kernel(int n, const float4* r, const float4* diag, float4* x,
                                                         float4* z, float4* p, double* partial) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    double rz = 0.0;
    if (v < n) {
        const float3 rv = f3(r[v]);
        const float3 zv = block_solve(diag[2 * v], diag[2 * v + 1], rv);
        x[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        z[v] = make_float4(zv.x, zv.y, zv.z, 0.f);
        p[v] = z[v];
        rz = (double)rv.x * zv.x + (double)rv.y * zv.y + (double)rv.z * zv.z;
    }
    block_partial(rz, partial);
}

__global__ void __launch_bounds__(kBlock) cg_update_kernel(int n, const double* sc, float4* x, float4* r,
                                                           const float4* p, const float4* q, const float4* diag,
                                                           float4* z, double* part_rz, double* part_rr,
                                                           int32_t* flag) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const double pq = sc[1];
    const bool stop = *flag != 0 || !(pq > 0.0);
    double rz = 0.0, rr = 0.0;
    if (!stop && v < n) {
        const float alpha = (float)(sc[0] / pq);
        const float4 xv = x[v], pv = p[v], qv = q[v];
        float3 rv = f3(r[v]);
        x[v] = make_float4(xv.x + alpha * pv.x, xv.y + alpha * pv.y, xv.z + alpha * pv.z, 0.f);
        rv = make_float3(rv.x - alpha * qv.x, rv.y - alpha * qv.y, rv.z - alpha * qv.z);
        r[v] = make_float4(rv.x, rv.y, rv.z, 0.f);
        const float3 zv = block_solve(diag[2 * v], diag[2 * v + 1], rv);
        z[v] = make_float4(zv.x, zv.y, zv.z, 0.f);
        rz = (double)rv.x * zv.x + (double)rv.y * zv.y + (double)rv.z * zv.z;
        rr = (double)rv.x * rv.x + (double)rv.y * rv.y + (double)rv.z * rv.z;
    }
    if (stop && v == 0 && *flag == 0) atomicOr(flag, 1);
    block_partial(rz, part_rz);
    block_partial(rr, part_rr);
}

__global__ void __launch_bounds__(kBlock) cg_dir_kernel(int n, const double* sc, const float4* z, float4* p,
                                                        const int32_t* flag) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || *flag) return;
    const float beta = (float)(sc[2] / sc[0]);
    const float4 zv = z[v], pv = p[v];
    p[v] = make_float4(zv.x + beta * pv.x, zv.y + beta * pv.y, zv.z + beta * pv.z, 0.f);
}

__global__ void cg_shift_kernel(double* sc, const int32_t* flag) {
    if (!*flag) sc[0] = sc[2];
}

// dst = src + s x on free vertices (compensated pairs); clamped vertices copied.
__global__ void newton_axpy_kernel(int nv, int nfree, State src, const float4* x, float s, State dst) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    float4 h = src.hi[v], l = src.lo[v];
    if (v < nfree) {
        const float4 xv = x[v];
        el::pair_add(h.x, l.x, s * xv.x);
        el::pair_add(h.y, l.y, s * xv.y);
        el::pair_add(h.z, l.z, s * xv.z);
    }
    dst.hi[v] = h;
    dst.lo[v] = l;
}

// Internal float4 vector (free rows, zero elsewhere) <-> caller float [nv][3].
__global__ void gather_vec_kernel(int nv, int nfree, const int32_t* perm, const float* in, float4* out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int o = perm[v];
    out[v] = v < nfree ? make_float4(in[3 * o], in[3 * o + 1], in[3 * o + 2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void scatter_vec_kernel(int nv, int nfree, const int32_t* perm, const float4* in, float* out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int o = perm[v];
    const float4 a = v < nfree ? in[v] : make_float4(0.f, 0.f, 0.f, 0.f);
    out[3 * o] = a.x;
    out[3 * o + 1] = a.y;
    out[3 * o + 2] = a.z;
}

}  // namespace

int adjoint_warps(int nitems) { return nblocks(nitems, kBlock / 32) * (kBlock / 32); }

template <int MODE, int MODEL>
cudaError_t vertex_launch(int grid, const DeviceMesh& m, State u, float4* lam, const float4* gv, float4* diag,
                          float4* out, const Item* items, int nitems, int32_t* err, double* partial, cudaStream_t st) {
    adjoint_vertex_kernel<MODE, MODEL><<<grid, kBlock, 0, st>>>(m, u, lam, gv, diag, out, items, nitems, err, partial);
    return cudaGetLastError();
}

template <int MODEL>
cudaError_t vertex_launch_model(int mode, int grid, const DeviceMesh& m, State u, float4* lam, const float4* gv,
                                float4* diag, float4* out, const Item* items, int nitems, int32_t* err,
                                double* partial, cudaStream_t st) {
    switch (mode) {
        case kDiag: return vertex_launch<kDiag, MODEL>(grid, m, u, lam, gv, diag, out, items, nitems, err, partial, st);
        case kSweep: return vertex_launch<kSweep, MODEL>(grid, m, u, lam, gv, diag, out, items, nitems, err, partial, st);
        case kResid: return vertex_launch<kResid, MODEL>(grid, m, u, lam, gv, diag, out, items, nitems, err, partial, st);
        case kForce: return vertex_launch<kForce, MODEL>(grid, m, u, lam, gv, diag, out, items, nitems, err, partial, st);
        default: return vertex_launch<kApply, MODEL>(grid, m, u, lam, gv, diag, out, items, nitems, err, partial, st);
    }
}

cudaError_t launch_adjoint_vertex(int mode, const DeviceMesh& m, State u, float4* lam, const float4* gv,
                                  float4* diag, const Item* items, int nitems, int32_t* err, double* partial,
                                  cudaStream_t st, float4* out, int model) {
    if (nitems <= 0) return cudaSuccess;
    const int grid = nblocks(nitems, kBlock / 32);
    if (model == el::kNeoHookean)
        return vertex_launch_model<el::kNeoHookean>(mode, grid, m, u, lam, gv, diag, out, items, nitems, err, partial, st);
    if (model == el::kStableNeoHookean)
        return vertex_launch_model<el::kStableNeoHookean>(mode, grid, m, u, lam, gv, diag, out, items, nitems, err,
                                                          partial, st);
    return vertex_launch_model<el::kCorotated>(mode, grid, m, u, lam, gv, diag, out, items, nitems, err, partial, st);
}

cudaError_t adjoint_prepare() {
    const int bytes = kAdjWarps * (int)sizeof(AdjWarpSmem);
    const void* fns[6] = {(const void*)adjoint_ring_sweep_kernel<el::kCorotated, false>,
                          (const void*)adjoint_ring_sweep_kernel<el::kNeoHookean, false>,
                          (const void*)adjoint_ring_sweep_kernel<el::kStableNeoHookean, false>,
                          (const void*)adjoint_ring_sweep_kernel<el::kCorotated, true>,
                          (const void*)adjoint_ring_sweep_kernel<el::kNeoHookean, true>,
                          (const void*)adjoint_ring_sweep_kernel<el::kStableNeoHookean, true>};
    for (const void* f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int adj_ring_grid(int nitems) {
    const int want = nblocks(nitems, kAdjWarps), cap = kAdjCtasPerSm * adj_sm_count();
    return want < cap ? want : cap;
}

template <bool APPLY>
cudaError_t adj_ring_launch(const DeviceMesh& m, State u, float4* lam, const float4* gv, const float4* diag,
                            const Item* items, int nitems, int32_t* err, int model, float4* out, double* partial,
                            cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const int bytes = kAdjWarps * (int)sizeof(AdjWarpSmem);  // attribute set by adjoint_prepare()
    const int grid = adj_ring_grid(nitems);
    if (model == el::kNeoHookean)
        adjoint_ring_sweep_kernel<el::kNeoHookean, APPLY><<<grid, kAdjWarps * 32, bytes, st>>>(
            m, u, lam, gv, diag, items, nitems, err, out, partial);
    else if (model == el::kStableNeoHookean)
        adjoint_ring_sweep_kernel<el::kStableNeoHookean, APPLY><<<grid, kAdjWarps * 32, bytes, st>>>(
            m, u, lam, gv, diag, items, nitems, err, out, partial);
    else
        adjoint_ring_sweep_kernel<el::kCorotated, APPLY><<<grid, kAdjWarps * 32, bytes, st>>>(
            m, u, lam, gv, diag, items, nitems, err, out, partial);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_ring_sweep(const DeviceMesh& m, State u, float4* lam, const float4* gv, const float4* diag,
                                      const Item* items, int nitems, int32_t* err, int model, cudaStream_t st) {
    return adj_ring_launch<false>(m, u, lam, gv, diag, items, nitems, err, model, nullptr, nullptr, st);
}

int adjoint_ring_apply_warps(int nitems) { return nitems > 0 ? adj_ring_grid(nitems) * kAdjWarps : 0; }

cudaError_t launch_adjoint_ring_apply(const DeviceMesh& m, State u, const float4* lam, const Item* items, int nitems,
                                      int32_t* err, int model, float4* out, double* partial, cudaStream_t st) {
    return adj_ring_launch<true>(m, u, const_cast<float4*>(lam), nullptr, nullptr, items, nitems, err, model, out,
                                 partial, st);
}

int vec_blocks(int n) { return nblocks(n, kBlock); }

cudaError_t launch_cg_init(int n, const float4* r, const float4* diag, float4* x, float4* z, float4* p,
                           double* partial, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cg_init_kernel<<<nblocks(n, kBlock), kBlock, 0, st>>>(n, r, diag, x, z, p, partial);
    return cudaGetLastError();
}

cudaError_t launch_cg_update(int n, const double* sc, float4* x, float4* r, const float4* p, const float4* q,
                             const float4* diag, float4* z, double* part_rz, double* part_rr, int32_t* flag,
                             cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cg_update_kernel<<<nblocks(n, kBlock), kBlock, 0, st>>>(n, sc, x, r, p, q, diag, z, part_rz, part_rr, flag);
    return cudaGetLastError();
}

cudaError_t launch_cg_dir(int n, const double* sc, const float4* z, float4* p, const int32_t* flag, double* sc_rw,
                          cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cg_dir_kernel<<<nblocks(n, kBlock), kBlock, 0, st>>>(n, sc, z, p, flag);
    cg_shift_kernel<<<1, 1, 0, st>>>(sc_rw, flag);
    return cudaGetLastError();
}

cudaError_t launch_newton_axpy(int nv, int nfree, State src, const float4* x, float s, State dst, cudaStream_t st) {
    if (nv <= 0) return cudaSuccess;
    newton_axpy_kernel<<<nblocks(nv, 256), 256, 0, st>>>(nv, nfree, src, x, s, dst);
    return cudaGetLastError();
}

cudaError_t launch_gather_vec(int nv, int nfree, const int32_t* perm, const float* in, float4* out, cudaStream_t st) {
    if (nv <= 0) return cudaSuccess;
    gather_vec_kernel<<<nblocks(nv, 256), 256, 0, st>>>(nv, nfree, perm, in, out);
    return cudaGetLastError();
}

cudaError_t launch_scatter_vec(int nv, int nfree, const int32_t* perm, const float4* in, float* out, cudaStream_t st) {
    if (nv <= 0) return cudaSuccess;
    scatter_vec_kernel<<<nblocks(nv, 256), 256, 0, st>>>(nv, nfree, perm, in, out);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_tets(int ne, int nfree, const int4* tv, const float4* tb, State u, const float4* lam,
                                float* dLdlogE, float* hdl, cudaStream_t st, int model) {
    if (ne <= 0) return cudaSuccess;
    const int grid = nblocks(ne, 128);
    if (model == el::kNeoHookean)
        adjoint_tet_kernel<el::kNeoHookean><<<grid, 128, 0, st>>>(ne, nfree, tv, tb, u, lam, dLdlogE, hdl);
    else if (model == el::kStableNeoHookean)
        adjoint_tet_kernel<el::kStableNeoHookean><<<grid, 128, 0, st>>>(ne, nfree, tv, tb, u, lam, dLdlogE, hdl);
    else
        adjoint_tet_kernel<el::kCorotated><<<grid, 128, 0, st>>>(ne, nfree, tv, tb, u, lam, dLdlogE, hdl);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_weak_clamped(int nwc, int nfree, const DeviceMesh& m, const float4* lam, float* hdl,
                                        cudaStream_t st) {
    if (nwc <= 0 || !m.wc_v) return cudaSuccess;
    adjoint_weak_clamped_kernel<<<nblocks(nwc, 256), 256, 0, st>>>(nwc, nfree, m, lam, hdl);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_shift(int nv, State u, const float4* lam_hi, const float4* lam_lo, float eps, State up,
                                 State um, cudaStream_t st) {
    if (nv <= 0) return cudaSuccess;
    adjoint_shift_kernel<<<nblocks(nv, 256), 256, 0, st>>>(nv, u, lam_hi, lam_lo, eps, up, um);
    return cudaGetLastError();
}

int adj_vec_blocks(int n) { return n > 0 ? nblocks(n, kVecBlock) : 0; }

cudaError_t launch_adjoint_refine_rhs(int nfree, const float4* gv, const float4* fp_hi, const float4* fp_lo,
                                      const float4* fm_hi, const float4* fm_lo, double inv2eps, float4* rhs,
                                      double* partial, cudaStream_t st) {
    if (nfree <= 0) return cudaSuccess;
    adjoint_refine_rhs_kernel<<<nblocks(nfree, kVecBlock), kVecBlock, 0, st>>>(nfree, gv, fp_hi, fp_lo, fm_hi, fm_lo,
                                                                                inv2eps, rhs, partial);
    return cudaGetLastError();
}

cudaError_t launch_acg_step(int n, const double* sc, int32_t* flag, const float4* p, const float4* q, float4* x,
                            float4* r, double* partial, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    acg_step_kernel<<<nblocks(n, kVecBlock), kVecBlock, 0, st>>>(n, sc, flag, p, q, x, r, partial);
    return cudaGetLastError();
}

cudaError_t launch_acg_dot(int n, const float4* r, const float4* z, double* partial, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    acg_dot_kernel<<<nblocks(n, kVecBlock), kVecBlock, 0, st>>>(n, r, z, partial);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_accumulate(int nfree, const float4* d, float4* lam_hi, float4* lam_lo, float* maxabs,
                                      cudaStream_t st) {
    if (nfree <= 0) return cudaSuccess;
    adjoint_accumulate_kernel<<<nblocks(nfree, 256), 256, 0, st>>>(nfree, d, lam_hi, lam_lo, maxabs);
    return cudaGetLastError();
}

cudaError_t launch_gather_rhs(int nfree, const int32_t* perm, const float* dLdu, float4* gv, cudaStream_t st) {
    if (nfree <= 0) return cudaSuccess;
    gather_rhs_kernel<<<nblocks(nfree, 256), 256, 0, st>>>(nfree, perm, dLdu, gv);
    return cudaGetLastError();
}

cudaError_t launch_clamped_grad(int nd, const int32_t* dq_internal, const int32_t* dq_caller, const float* dLdu,
                                const float* hdl, float* out, cudaStream_t st) {
    if (nd <= 0) return cudaSuccess;
    clamped_grad_kernel<<<nblocks(nd, 256), 256, 0, st>>>(nd, dq_internal, dq_caller, dLdu, hdl, out);
    return cudaGetLastError();
}

}  // namespace pbng
