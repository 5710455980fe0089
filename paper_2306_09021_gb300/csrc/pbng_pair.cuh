// The element term of the PBNG node update (pbng_element.cuh,
// element_math_m) for two tetrahedra at once in packed f32x2 arithmetic:
// every value is a float2 whose .x belongs to one tet and .y to the other,
// and each add, multiply or fused multiply-add on it is one packed
// instruction (sm_100 and later), so the float32 colour passes issue about
// half the floating-point instructions per tet.  The arithmetic per tet is
// the scalar version's, with its fused multiply-adds written out.
#pragma once

#include "pbng_element.cuh"

namespace pbng {
namespace pk {

__device__ __forceinline__ float2 sp(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __fadd2_rn(a, neg(b)); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a b - c
__device__ __forceinline__ float2 fms(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, neg(c)); }
// c - a b
__device__ __forceinline__ float2 fnms(float2 a, float2 b, float2 c) { return __ffma2_rn(neg(a), b, c); }
// a b - c d
__device__ __forceinline__ float2 dif(float2 a, float2 b, float2 c, float2 d) { return fms(a, b, mul(c, d)); }
// a0 b0 + a1 b1 + a2 b2
__device__ __forceinline__ float2 dot3(float2 a0, float2 b0, float2 a1, float2 b1, float2 a2, float2 b2) {
    return fma(a0, b0, fma(a1, b1, mul(a2, b2)));
}

// One Newton step's convergence test of polar_quaternion for one tet:
// converged, or quadratic convergence has set in and the step is below
// 1e-4 t (see there).
__device__ __forceinline__ bool newton_done(float ad, float t, float dprev) {
    return !(ad > 2e-7f * t) || (ad <= 1e-4f * t && ad <= 0.01f * dprev);
}

// polar_quaternion (pbng_element.cuh) for two tets: the largest root t of
// the characteristic polynomial of N by Newton from sqrt(3)|F|, column 0 of
// adj(N - t I), the best-scaled column where column 0 is not, normalised to
// length `scale`.  A tet whose iteration has converged keeps its t while the
// other's goes on.
__device__ __forceinline__ void polar_quaternion_pair(const float2* H, float2 n2, float2 c2, float2 J, float scale,
                                                      float2* qo) {
    const float2 k0 = fms(n2, n2, mul(sp(4.0f), c2));
    const float2 n23 = mul(sp(3.0f), n2);
    float2 t = make_float2(n23.x * rsqrtf(n23.x), n23.y * rsqrtf(n23.y));
    const float2 m8J = mul(sp(-8.0f), J), m2n2 = mul(sp(-2.0f), n2), m4n2 = mul(sp(-4.0f), n2);
    float2 dp = sp(1.0f);
    float dpx = 3e-3f * t.x, dpy = 3e-3f * t.y;  // previous steps, as in polar_quaternion
    bool dx = false, dy = false;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
        const float2 t2 = mul(t, t);
        const float2 p = fma(fma(add(t2, m2n2), t, m8J), t, k0);
        const float2 dpn = fma(fma(sp(4.0f), t2, m4n2), t, m8J);
        const float2 d = make_float2(__fdividef(p.x, dpn.x), __fdividef(p.y, dpn.y));
        const float2 tn = sub(t, d);
        if (!dx) {
            t.x = tn.x;
            dp.x = dpn.x;
            const float ad = fabsf(d.x);
            dx = newton_done(ad, t.x, dpx);
            dpx = ad;
        }
        if (!dy) {
            t.y = tn.y;
            dp.y = dpn.y;
            const float ad = fabsf(d.y);
            dy = newton_done(ad, t.y, dpy);
            dpy = ad;
        }
        if (dx && dy) break;
    }
    const float2 trH = add(add(H[0], H[4]), H[8]);
    const float2 m00 = add(sub(sp(3.0f), t), trH);
    const float2 mt = sub(sp(-1.0f), t);
    const float2 m11 = add(mt, sub(sub(H[0], H[4]), H[8]));
    const float2 m22 = add(mt, sub(sub(H[4], H[0]), H[8]));
    const float2 m33 = add(mt, sub(sub(H[8], H[0]), H[4]));
    const float2 m01 = sub(H[7], H[5]), m02 = sub(H[2], H[6]), m03 = sub(H[3], H[1]);
    const float2 m12 = add(H[1], H[3]), m13 = add(H[2], H[6]), m23 = add(H[5], H[7]);
    const float2 k01 = dif(m02, m13, m12, m03), k02 = dif(m02, m23, m22, m03), k03 = dif(m02, m33, m23, m03);
    const float2 k12 = dif(m12, m23, m22, m13), k13 = dif(m12, m33, m23, m13), k23 = dif(m22, m33, m23, m23);
    float2 q[4];
    q[0] = fma(m13, k12, fnms(m12, k13, mul(m11, k23)));
    q[1] = fnms(m01, k23, fms(m12, k03, mul(m13, k02)));
    q[2] = fma(m01, k13, fnms(m11, k03, mul(m13, k01)));
    q[3] = fnms(m01, k12, fms(m11, k02, mul(m12, k01)));
    if (!(-q[0].x > 0.25f * dp.x)) {
        float qs[4] = {q[0].x, q[1].x, q[2].x, q[3].x};
        el::adjugate_best_column(m00.x, m01.x, m02.x, m03.x, m11.x, m12.x, m13.x, m22.x, m23.x, m33.x, qs);
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k].x = qs[k];
    }
    if (!(-q[0].y > 0.25f * dp.y)) {
        float qs[4] = {q[0].y, q[1].y, q[2].y, q[3].y};
        el::adjugate_best_column(m00.y, m01.y, m02.y, m03.y, m11.y, m12.y, m13.y, m22.y, m23.y, m33.y, qs);
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k].y = qs[k];
    }
    const float2 qq = fma(q[0], q[0], fma(q[1], q[1], fma(q[2], q[2], mul(q[3], q[3]))));
    const bool okx = qq.x > 1e-30f && qq.x < 3.0e38f, oky = qq.y > 1e-30f && qq.y < 3.0e38f;
    const float2 inv = make_float2(okx ? scale * rsqrtf(qq.x) : 0.0f, oky ? scale * rsqrtf(qq.y) : 0.0f);
#pragma unroll
    for (int k = 0; k < 4; ++k) qo[k] = mul(q[k], inv);
    if (!okx) qo[0].x = scale;
    if (!oky) qo[0].y = scale;
}

// element_math_m (pbng_element.cuh) for two tets: gk = dN_jk/dX of the other
// three vertices, a = 2 mu V, b = lambda V, dk = u_jk - u_i, each component a
// (tet A, tet B) pair.  Writes V P(F) s with s = g_j1 + g_j2 + g_j3 (the
// vertex's force is the sum of these) to f and, with NEED_A, the modified
// Hessian of Eq. mod_hess_dens (upper triangle) to A.
template <bool NEED_A, int MODEL>
__device__ __forceinline__ void element_math_pair(const float2* g1, const float2* g2, const float2* g3, float2 a,
                                                  float2 b, const float2* d1, const float2* d2, const float2* d3,
                                                  float2* f, float2* A) {
    float2 H[9];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) H[3 * p + q] = dot3(d1[p], g1[q], d2[p], g2[q], d3[p], g3[q]);
    float2 s[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) s[q] = add(add(g1[q], g2[q]), g3[q]);
    const float2 one = sp(1.0f);
    const float2 F0 = add(one, H[0]), F4 = add(one, H[4]), F8 = add(one, H[8]);
    const float2 F1 = H[1], F2 = H[2], F3 = H[3], F5 = H[5], F6 = H[6], F7 = H[7];
    float2 C[9];
    C[0] = dif(F4, F8, F5, F7);
    C[1] = dif(F5, F6, F3, F8);
    C[2] = dif(F3, F7, F4, F6);
    C[3] = dif(F7, F2, F8, F1);
    C[4] = dif(F8, F0, F6, F2);
    C[5] = dif(F6, F1, F7, F0);
    C[6] = dif(F1, F5, F2, F4);
    C[7] = dif(F2, F3, F0, F5);
    C[8] = dif(F0, F4, F1, F3);
    // J - 1 = tr H + (sum of principal 2x2 minors of H) + det H
    const float2 trH = add(add(H[0], H[4]), H[8]);
    const float2 minors = sub(fma(H[0], H[4], fma(H[0], H[8], mul(H[4], H[8]))),
                              fma(H[1], H[3], fma(H[2], H[6], mul(H[5], H[7]))));
    const float2 c0 = dif(H[4], H[8], H[5], H[7]), c1 = dif(H[3], H[8], H[5], H[6]), c2h = dif(H[3], H[7], H[4], H[6]);
    const float2 detH = fma(H[0], c0, fnms(H[1], c1, mul(H[2], c2h)));
    const float2 Jm1 = add(add(trH, minors), detH);
    float2 ws[3], Hs[3];  // cof(F) s = -w, H s
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        ws[p] = dot3(C[3 * p], s[0], C[3 * p + 1], s[1], C[3 * p + 2], s[2]);
        Hs[p] = dot3(H[3 * p], s[0], H[3 * p + 1], s[1], H[3 * p + 2], s[2]);
    }
    const float2 bJ = mul(b, Jm1);
    if (MODEL == el::kCorotated) {
        const float2 Fm[9] = {F0, F1, F2, F3, F4, F5, F6, F7, F8};
        float2 n2 = mul(Fm[0], Fm[0]), c2 = mul(C[0], C[0]);
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            n2 = fma(Fm[k], Fm[k], n2);
            c2 = fma(C[k], C[k], c2);
        }
        float2 q[4];
        polar_quaternion_pair(H, n2, c2, add(one, Jm1), 1.41421356237309505f, q);
        const float2 x = q[1], y = q[2], z = q[3];
        const float2 cr[3] = {dif(y, s[2], z, s[1]), dif(z, s[0], x, s[2]), dif(x, s[1], y, s[0])};
        const float2 vs = dot3(x, s[0], y, s[1], z, s[2]);
        const float2 vv = dot3(x, x, y, y, z, z);
        const float2 vq[3] = {x, y, z};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            // (R - I) s = w (v x s) + v (v . s) - |v|^2 s
            const float2 rs = fma(q[0], cr[p], dif(vq[p], vs, vv, s[p]));
            f[p] = fma(a, sub(Hs[p], rs), mul(bJ, ws[p]));
        }
    } else {
        // cof(H), then (F - C) s = H s + H^T s - tr(H) s - cof(H) s
        float2 K[9];
        K[0] = dif(H[4], H[8], H[5], H[7]);
        K[1] = dif(H[5], H[6], H[3], H[8]);
        K[2] = dif(H[3], H[7], H[4], H[6]);
        K[3] = dif(H[7], H[2], H[8], H[1]);
        K[4] = dif(H[8], H[0], H[6], H[2]);
        K[5] = dif(H[6], H[1], H[7], H[0]);
        K[6] = dif(H[1], H[5], H[2], H[4]);
        K[7] = dif(H[2], H[3], H[0], H[5]);
        K[8] = dif(H[0], H[4], H[1], H[3]);
        const float2 ha = mul(sp(0.5f), a);
        float2 qs = sp(0.0f), kv = add(ha, b);
        if (MODEL == el::kStableNeoHookean) {
            float2 hh = mul(H[0], H[0]);
#pragma unroll
            for (int k = 1; k < 9; ++k) hh = fma(H[k], H[k], hh);
            const float2 ic3 = fma(sp(2.0f), trH, hh);  // I_C - 3
            const float2 ratio = make_float2(__fdividef(ic3.x, 4.0f + ic3.x), __fdividef(ic3.y, 4.0f + ic3.y));
            qs = mul(mul(a, sp(1.0f / 6.0f)), ratio);
            kv = fma(a, sp(5.0f / 12.0f), b);
        }
        const float2 kJ = mul(kv, Jm1);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float2 Hts = dot3(H[p], s[0], H[3 + p], s[1], H[6 + p], s[2]);
            const float2 Ks = dot3(K[3 * p], s[0], K[3 * p + 1], s[1], K[3 * p + 2], s[2]);
            const float2 fcs = sub(fnms(trH, s[p], add(Hs[p], Hts)), Ks);
            float2 t = fma(ha, fcs, mul(kJ, ws[p]));
            if (MODEL == el::kStableNeoHookean) t = fma(qs, add(s[p], Hs[p]), t);
            f[p] = t;
        }
    }
    if (NEED_A) {
        const float2 ag = mul(a, dot3(s[0], s[0], s[1], s[1], s[2], s[2]));
        const float2 bw0 = mul(b, ws[0]), bw1 = mul(b, ws[1]), bw2 = mul(b, ws[2]);
        A[0] = fma(bw0, ws[0], ag);
        A[1] = mul(bw0, ws[1]);
        A[2] = mul(bw0, ws[2]);
        A[3] = fma(bw1, ws[1], ag);
        A[4] = mul(bw1, ws[2]);
        A[5] = fma(bw2, ws[2], ag);
    }
}

}  // namespace pk
}  // namespace pbng
