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

// A running sum of float-float terms and products (Ogita, Rump and Oishi's
// Sum2 / Dot2, 2005): the high words are summed by TwoSum into s, every
// rounding error and every low-order part (the low words and the cross
// products of a float-float product) into the float c.  The value s + c is
// as accurate as if the sum had been formed with twice the precision, and is
// normalised once, at the end, instead of after every term.
struct Acc {
    float s, c;
};
PBNG_FF_HD Acc acc_of(F2 x) { return Acc{x.h, x.l}; }
// x y, exactly up to the low words' product
PBNG_FF_HD Acc acc_prod(F2 x, F2 y) {
    const float p = fmul(x.h, y.h);
    return Acc{p, ffma(x.h, y.l, ffma(x.l, y.h, ffma(x.h, y.h, -p)))};
}
PBNG_FF_HD void acc_add(Acc& a, F2 x) {
    const F2 t = two_sum(a.s, x.h);
    a.s = t.h;
    a.c = fadd(a.c, fadd(t.l, x.l));
}
PBNG_FF_HD void acc_add(Acc& a, float x) {
    const F2 t = two_sum(a.s, x);
    a.s = t.h;
    a.c = fadd(a.c, t.l);
}
// a += x y
PBNG_FF_HD void acc_fma(Acc& a, F2 x, F2 y) {
    const float p = fmul(x.h, y.h);
    const float e = ffma(x.h, y.h, -p);
    const F2 t = two_sum(a.s, p);
    a.s = t.h;
    a.c = ffma(x.h, y.l, ffma(x.l, y.h, fadd(a.c, fadd(t.l, e))));
}
// a += x y for a float y
PBNG_FF_HD void acc_fma(Acc& a, F2 x, float y) {
    const float p = fmul(x.h, y);
    const float e = ffma(x.h, y, -p);
    const F2 t = two_sum(a.s, p);
    a.s = t.h;
    a.c = ffma(x.l, y, fadd(a.c, fadd(t.l, e)));
}
// s + c as a normalised pair (TwoSum: c may exceed s where the terms cancel)
PBNG_FF_HD F2 acc_val(Acc a) { return two_sum(a.s, a.c); }
// x0 y0 + x1 y1 + x2 y2
PBNG_FF_HD F2 dot3(F2 x0, F2 y0, F2 x1, F2 y1, F2 x2, F2 y2) {
    Acc a = acc_prod(x0, y0);
    acc_fma(a, x1, y1);
    acc_fma(a, x2, y2);
    return acc_val(a);
}
// a b - c d
PBNG_FF_HD F2 dif2(F2 a, F2 b, F2 c, F2 d) {
    Acc t = acc_prod(a, b);
    acc_fma(t, neg(c), d);
    return acc_val(t);
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
        for (int c = 0; c < 3; ++c) H[3 * p + c] = dot3(d[0][p], g[0][c], d[1][p], g[1][c], d[2][p], g[2][c]);
    F2 s[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Acc t = acc_of(g[0][c]);
        acc_add(t, g[1][c]);
        acc_add(t, g[2][c]);
        s[c] = acc_val(t);
    }
    F2 F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = H[k];
    F[0] = add(F[0], 1.0f);
    F[4] = add(F[4], 1.0f);
    F[8] = add(F[8], 1.0f);
    // cofactor matrix C = det(F) F^{-T}
    F2 C[9];
    C[0] = dif2(F[4], F[8], F[5], F[7]);
    C[1] = dif2(F[5], F[6], F[3], F[8]);
    C[2] = dif2(F[3], F[7], F[4], F[6]);
    C[3] = dif2(F[7], F[2], F[8], F[1]);
    C[4] = dif2(F[8], F[0], F[6], F[2]);
    C[5] = dif2(F[6], F[1], F[7], F[0]);
    C[6] = dif2(F[1], F[5], F[2], F[4]);
    C[7] = dif2(F[2], F[3], F[0], F[5]);
    C[8] = dif2(F[0], F[4], F[1], F[3]);
    Acc jacc = acc_prod(F[0], C[0]);
    acc_fma(jacc, F[1], C[1]);
    acc_fma(jacc, F[2], C[2]);
    acc_add(jacc, -1.0f);
    const F2 Jm1 = acc_val(jacc);  // det F - 1
    F2 ws[3], Hs[3];  // C s, H s
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        ws[p] = dot3(C[3 * p], s[0], C[3 * p + 1], s[1], C[3 * p + 2], s[2]);
        Hs[p] = dot3(H[3 * p], s[0], H[3 * p + 1], s[1], H[3 * p + 2], s[2]);
    }
    F2 f[3];
    if (MODEL == kCorotated) {
        // R0 = I + K0 from the quaternion, exactly orthogonal up to
        // float-float rounding: K0 = 2 (w [v]x + [v]x^2) / |q|^2.
        const float w = q[0], x = q[1], y = q[2], z = q[3];
        Acc qa = acc_prod(mk(w), mk(w));
        acc_fma(qa, mk(x), x);
        acc_fma(qa, mk(y), y);
        acc_fma(qa, mk(z), z);
        const F2 inv2 = mul(recip(acc_val(qa)), 2.0f);
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
        // M = R0^T F = I + K0^T + H + K0^T H, M_rc = K[3c + r] + H[3r + c] +
        // sum_k K[3k + r] H[3k + c].  Its skew part (float-float, each
        // difference M_rc - M_cr in one running sum) gives the correction;
        // its symmetric part S only needs float.
        auto skew = [&](int r, int c) -> float {  // M_rc - M_cr
            Acc t = acc_of(K[3 * c + r]);
            acc_add(t, H[3 * r + c]);
            acc_add(t, neg(K[3 * r + c]));
            acc_add(t, neg(H[3 * c + r]));
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                acc_fma(t, K[3 * k + r], H[3 * k + c]);
                acc_fma(t, neg(K[3 * k + c]), H[3 * k + r]);
            }
            return fadd(t.s, t.c);
        };
        const float ax = 0.5f * skew(2, 1), ay = 0.5f * skew(0, 2), az = 0.5f * skew(1, 0);
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
            // a (H s - (R - I) s) + b (J - 1) C s with (R - I) s = K0 s + corr;
            // H s and K0 s nearly cancel (the rotation), so their difference
            // is formed first
            const F2 Ks = dot3(K[3 * p], s[0], K[3 * p + 1], s[1], K[3 * p + 2], s[2]);
            Acc dd = acc_of(Hs[p]);
            acc_add(dd, neg(Ks));
            acc_add(dd, -corr);
            Acc t = acc_prod(a, acc_val(dd));
            acc_fma(t, bJ, ws[p]);
            f[p] = acc_val(t);
        }
    } else {
        // (F - C) s = s + H s - C s
        const F2 ha = mul(a, 0.5f);
        F2 kv = add(ha, b);
        F2 qs = mk(0.0f);
        if (MODEL == kStableNeoHookean) {
            Acc hh = acc_prod(H[0], H[0]);
#pragma unroll
            for (int k = 1; k < 9; ++k) acc_fma(hh, H[k], H[k]);
            acc_fma(hh, H[0], 2.0f);
            acc_fma(hh, H[4], 2.0f);
            acc_fma(hh, H[8], 2.0f);
            const F2 ic3 = acc_val(hh);  // I_C - 3 = 2 tr H + |H|^2
            // 1/6 and 5/12 are not floats: their float-pair values
            qs = mul(div(ic3, add(ic3, 4.0f)), mul(a, mk(0.16666667163f, -4.9670539e-9f)));
            kv = add(b, mul(a, mk(0.4166666567f, 9.9341078e-9f)));
        }
        const F2 kJ = mul(kv, Jm1);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            // (F - C) s = s + H s - C s, which cancels near F = I, first
            Acc fc = acc_of(s[p]);
            acc_add(fc, Hs[p]);
            const F2 sh = acc_val(fc);  // F s
            acc_add(fc, neg(ws[p]));
            Acc t = acc_prod(ha, acc_val(fc));
            acc_fma(t, kJ, ws[p]);
            if (MODEL == kStableNeoHookean) acc_fma(t, qs, sh);
            f[p] = acc_val(t);
        }
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) fout[p] = f[p];
}

}  // namespace ff
}  // namespace pbng
