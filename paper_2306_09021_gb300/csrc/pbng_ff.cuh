// Extended-precision element force for the residual and for the update
// passes of PBNG_PREC_EXTENDED.
//
// Near an equilibrium the nodal force f_i + f^ext_i is a small sum of
// per-element terms V P(F) g_i that are far larger than it: on a 64^3 cube
// under gravity each term is about 180 times the nodal load.  A float32
// evaluation (or float32 element constants) leaves an error of about 1e-7 of
// each term in the sum, which bounds the relative residual that can be
// measured or reached to about 1e-4.  Here each term is evaluated in
// float-float arithmetic (a value is an unevaluated sum h + l of two floats,
// about 48 significant bits) from float-pair element constants and the
// float-pair iterate, and the caller sums the terms in float-float too.
//
// Float-float operations follow Dekker (1971) and Knuth's TwoSum: an exact
// product by FMA, an exact sum by TwoSum, and the low words of the operands
// added in with one rounding.  Their error is about 2^-47 of the larger
// operand, which is what the cancelling sums need.
//
// The polar rotation R of Eq. cor is taken from a float32 quaternion
// estimate (accurate to a few ulp) and refined once: with R0 the rotation of
// the quaternion (formed in float-float, so it is orthogonal to float-float
// accuracy) and M = R0^T F, the rotation R = R0 exp([theta]x) that makes
// R^T F symmetric has, to first order in the small theta,
//   (tr(S) I - S) theta = 2 axial(skew(M)),   S = sym(M)
// (from [t]x S + S [t]x = [(tr(S) I - S) t]x for symmetric S).  The error
// after the step is of the order of theta squared, below float-float
// resolution.
//
// Everything is __host__ __device__ so that the same arithmetic can be
// checked on a CPU.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define PBNG_FF_HD __host__ __device__ __forceinline__
#else
#define PBNG_FF_HD inline
#endif

namespace pbng {
namespace ff {

// Correctly rounded float operations that the compiler may not contract
// into FMAs (the error-free transformations depend on it).
PBNG_FF_HD float fadd(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    volatile float s = a + b;
    return s;
#endif
}
PBNG_FF_HD float fmul(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    volatile float p = a * b;
    return p;
#endif
}
PBNG_FF_HD float ffma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}

struct F2 {
    float h, l;
};

PBNG_FF_HD F2 mk(float h) { return F2{h, 0.0f}; }
PBNG_FF_HD F2 mk(float h, float l) { return F2{h, l}; }
PBNG_FF_HD double to_d(F2 a) { return (double)a.h + (double)a.l; }
PBNG_FF_HD F2 neg(F2 a) { return F2{-a.h, -a.l}; }

// a + b = s + e exactly (Knuth).
PBNG_FF_HD F2 two_sum(float a, float b) {
    const float s = fadd(a, b);
    const float bb = fadd(s, -a);
    const float e = fadd(fadd(a, -fadd(s, -bb)), fadd(b, -bb));
    return F2{s, e};
}
// a + b = s + e exactly when |a| >= |b| or a == 0 (Dekker).
PBNG_FF_HD F2 quick_two_sum(float a, float b) {
    const float s = fadd(a, b);
    return F2{s, fadd(b, -fadd(s, -a))};
}
// a b = p + e exactly (FMA).
PBNG_FF_HD F2 two_prod(float a, float b) {
    const float p = fmul(a, b);
    return F2{p, ffma(a, b, -p)};
}

// The low words are added with one rounding (Dekker's "sloppy" sum): the
// error is about 2^-48 of the larger operand, relative accuracy of the
// result is lost only where the high words cancel, which is the absolute
// accuracy these sums need.
PBNG_FF_HD F2 add(F2 a, F2 b) {
    const F2 s = two_sum(a.h, b.h);
    return quick_two_sum(s.h, fadd(s.l, fadd(a.l, b.l)));
}
PBNG_FF_HD F2 add(F2 a, float b) {
    const F2 s = two_sum(a.h, b);
    return quick_two_sum(s.h, fadd(s.l, a.l));
}
PBNG_FF_HD F2 sub(F2 a, F2 b) { return add(a, neg(b)); }
PBNG_FF_HD F2 mul(F2 a, F2 b) {
    const F2 p = two_prod(a.h, b.h);
    return quick_two_sum(p.h, ffma(a.h, b.l, ffma(a.l, b.h, p.l)));
}
PBNG_FF_HD F2 mul(F2 a, float b) {
    const F2 p = two_prod(a.h, b);
    return quick_two_sum(p.h, ffma(a.l, b, p.l));
}
// a b - c d with one normalisation.
PBNG_FF_HD F2 mul_sub(F2 a, F2 b, F2 c, F2 d) { return sub(mul(a, b), mul(c, d)); }
// 1 / a: Newton correction of the float reciprocal.
PBNG_FF_HD F2 recip(F2 a) {
    const float r = 1.0f / a.h;
    const F2 e = add(neg(mul(a, r)), 1.0f);  // 1 - a r
    return add(mk(r), e.h * r);
}
// a / b: float quotient, then the correction from the float-float remainder.
PBNG_FF_HD F2 div(F2 a, F2 b) {
    const float q = a.h / b.h;
    const F2 rem = sub(a, mul(b, q));
    return add(mk(q), rem.h / b.h);
}

// y = M x for a row-major float-float 3x3 and a float-float 3-vector.
PBNG_FF_HD void matvec(const F2* M, const F2* x, F2* y) {
#pragma unroll
    for (int p = 0; p < 3; ++p) y[p] = add(add(mul(M[3 * p], x[0]), mul(M[3 * p + 1], x[1])), mul(M[3 * p + 2], x[2]));
}

enum { kCorotated = 0, kNeoHookean = 1, kStableNeoHookean = 2 };

// f = V P(F) s of one element, with s = -g_i = g_j1 + g_j2 + g_j3 and
// F = I + H, H = sum_k d_k g_jk^T (Section "Discretization": the P1
// deformation gradient from the displacement differences d_k = u_jk - u_i).
//   g[k][c]  dN_jk/dX (float pairs), a = 2 mu V, b = lambda V (float pairs)
//   d[k][c]  displacement differences (float pairs)
//   q        float32 quaternion estimate (w, x, y, z) of the polar rotation,
//            any positive scale (corotated only)
// P is Eq. cor (corotated), Eq. nh (Neo-Hookean, lambda_hat = mu + lambda),
// or Eq. snh with lambda' on its volume term and the Lame reparametrisation
// mu' = 4mu/3, lambda' = lambda + 5mu/6 (stable Neo-Hookean), as in the
// float32 element term.  Writes f as float pairs.
template <int MODEL>
PBNG_FF_HD void element_force(const F2 g[3][3], F2 a, F2 b, const F2 d[3][3], const float* q, F2* fout) {
    F2 H[9];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            H[3 * p + c] = add(add(mul(d[0][p], g[0][c]), mul(d[1][p], g[1][c])), mul(d[2][p], g[2][c]));
    F2 s[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) s[c] = add(add(g[0][c], g[1][c]), g[2][c]);
    F2 F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = H[k];
    F[0] = add(F[0], 1.0f);
    F[4] = add(F[4], 1.0f);
    F[8] = add(F[8], 1.0f);
    // cofactor matrix C = det(F) F^{-T}
    F2 C[9];
    C[0] = mul_sub(F[4], F[8], F[5], F[7]);
    C[1] = mul_sub(F[5], F[6], F[3], F[8]);
    C[2] = mul_sub(F[3], F[7], F[4], F[6]);
    C[3] = mul_sub(F[7], F[2], F[8], F[1]);
    C[4] = mul_sub(F[8], F[0], F[6], F[2]);
    C[5] = mul_sub(F[6], F[1], F[7], F[0]);
    C[6] = mul_sub(F[1], F[5], F[2], F[4]);
    C[7] = mul_sub(F[2], F[3], F[0], F[5]);
    C[8] = mul_sub(F[0], F[4], F[1], F[3]);
    const F2 J = add(add(mul(F[0], C[0]), mul(F[1], C[1])), mul(F[2], C[2]));
    const F2 Jm1 = add(J, -1.0f);
    F2 ws[3], Hs[3];  // C s, H s
    matvec(C, s, ws);
    matvec(H, s, Hs);
    F2 f[3];
    if (MODEL == kCorotated) {
        // R0 = I + K0 from the quaternion, exactly orthogonal up to
        // float-float rounding: K0 = 2 (w [v]x + [v]x^2) / |q|^2.
        const float w = q[0], x = q[1], y = q[2], z = q[3];
        const F2 qq = add(add(two_prod(w, w), two_prod(x, x)), add(two_prod(y, y), two_prod(z, z)));
        const F2 inv2 = mul(recip(qq), 2.0f);
        const F2 xx = two_prod(x, x), yy = two_prod(y, y), zz = two_prod(z, z);
        const F2 xy = two_prod(x, y), xz = two_prod(x, z), yz = two_prod(y, z);
        const F2 wx = two_prod(w, x), wy = two_prod(w, y), wz = two_prod(w, z);
        F2 K[9];
        K[0] = mul(neg(add(yy, zz)), inv2);
        K[1] = mul(sub(xy, wz), inv2);
        K[2] = mul(add(xz, wy), inv2);
        K[3] = mul(add(xy, wz), inv2);
        K[4] = mul(neg(add(xx, zz)), inv2);
        K[5] = mul(sub(yz, wx), inv2);
        K[6] = mul(sub(xz, wy), inv2);
        K[7] = mul(add(yz, wx), inv2);
        K[8] = mul(neg(add(xx, yy)), inv2);
        // M = R0^T F = I + K0^T + H + K0^T H.  Its skew part (float-float)
        // gives the correction; its symmetric part S only needs float.
        auto mentry = [&](int r, int c) -> F2 {  // (K0^T + H + K0^T H)_rc
            F2 t = add(K[3 * c + r], H[3 * r + c]);
            t = add(t, mul(K[r], H[c]));
            t = add(t, mul(K[3 + r], H[3 + c]));
            return add(t, mul(K[6 + r], H[6 + c]));
        };
        const F2 m01 = mentry(0, 1), m10 = mentry(1, 0), m02 = mentry(0, 2), m20 = mentry(2, 0);
        const F2 m12 = mentry(1, 2), m21 = mentry(2, 1);
        const float ax = 0.5f * sub(m21, m12).h, ay = 0.5f * sub(m02, m20).h, az = 0.5f * sub(m10, m01).h;
        // S = sym(M) in float: I + sym(K0^T + H + K0^T H)
        float S[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                S[3 * r + c] = K[3 * c + r].h + H[3 * r + c].h + K[r].h * H[c].h + K[3 + r].h * H[3 + c].h +
                               K[6 + r].h * H[6 + c].h;
            }
        float Ss[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Ss[3 * r + c] = 0.5f * (S[3 * r + c] + S[3 * c + r]) + (r == c ? 1.0f : 0.0f);
        const float tr = Ss[0] + Ss[4] + Ss[8];
        // G = tr(S) I - S, theta = 2 G^{-1} axial(skew M) (adjugate solve)
        const float G0 = tr - Ss[0], G1 = -Ss[1], G2 = -Ss[2], G4 = tr - Ss[4], G5 = -Ss[5], G8 = tr - Ss[8];
        const float c00 = G4 * G8 - G5 * G5, c01 = G2 * G5 - G1 * G8, c02 = G1 * G5 - G2 * G4;
        const float c11 = G0 * G8 - G2 * G2, c12 = G1 * G2 - G0 * G5, c22 = G0 * G4 - G1 * G1;
        const float det = G0 * c00 + G1 * c01 + G2 * c02;
        float th[3] = {0.0f, 0.0f, 0.0f};
        if (fabsf(det) > 1e-6f * tr * tr * tr) {
            const float sc = 2.0f / det;
            th[0] = sc * (c00 * ax + c01 * ay + c02 * az);
            th[1] = sc * (c01 * ax + c11 * ay + c12 * az);
            th[2] = sc * (c02 * ax + c12 * ay + c22 * az);
        }
        // (R - I) s = K0 s + R0 (theta x s + theta x (theta x s) / 2); the
        // second term is of the order of the float32 rotation error, so float
        // suffices for it.
        F2 Ks[3];
        matvec(K, s, Ks);
        const float t1x = th[1] * s[2].h - th[2] * s[1].h;
        const float t1y = th[2] * s[0].h - th[0] * s[2].h;
        const float t1z = th[0] * s[1].h - th[1] * s[0].h;
        const float tsx = t1x + 0.5f * (th[1] * t1z - th[2] * t1y);
        const float tsy = t1y + 0.5f * (th[2] * t1x - th[0] * t1z);
        const float tsz = t1z + 0.5f * (th[0] * t1y - th[1] * t1x);
        const F2 bJ = mul(b, Jm1);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float corr = (K[3 * p].h * tsx + K[3 * p + 1].h * tsy + K[3 * p + 2].h * tsz) +
                               (p == 0 ? tsx : (p == 1 ? tsy : tsz));
            const F2 rs = add(Ks[p], corr);
            f[p] = add(mul(a, sub(Hs[p], rs)), mul(bJ, ws[p]));
        }
    } else {
        // (F - C) s = s + H s - C s
        const F2 ha = mul(a, 0.5f);
        F2 kv = add(ha, b);
        F2 qs = mk(0.0f);
        if (MODEL == kStableNeoHookean) {
            F2 hh = mk(0.0f);
#pragma unroll
            for (int k = 0; k < 9; ++k) hh = add(hh, mul(H[k], H[k]));
            const F2 trH = add(add(H[0], H[4]), H[8]);
            const F2 ic3 = add(mul(trH, 2.0f), hh);  // I_C - 3
            // 1/6 and 5/12 are not floats: their float-pair values
            qs = mul(div(ic3, add(ic3, 4.0f)), mul(a, mk(0.16666667163f, -4.9670539e-9f)));
            kv = add(b, mul(a, mk(0.4166666567f, 9.9341078e-9f)));
        }
        const F2 kJ = mul(kv, Jm1);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const F2 fcs = sub(add(s[p], Hs[p]), ws[p]);
            F2 t = add(mul(ha, fcs), mul(kJ, ws[p]));
            if (MODEL == kStableNeoHookean) t = add(t, mul(qs, add(s[p], Hs[p])));
            f[p] = t;
        }
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) fout[p] = f[p];
}

}  // namespace ff
}  // namespace pbng
