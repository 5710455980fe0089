// CUDA kernels of the PBNG sweep for sm_103a.
//
// One colour pass updates every free vertex of one colour (Section "Coloring
// and Parallelism"): a group of W lanes of one warp owns a vertex, each lane
// takes incident tetrahedra from the vertex's contiguous run of per-incidence
// records, forms the element's contribution to the nodal force and to the
// modified Hessian (Section "Modified Hessian", Eq. mod_hess), the group sums
// them with warp shuffles, and the group's first lane adds the weak/contact
// terms (Section "Weak Constraints"), solves the 3x3 system of Eq. pbgn_dx
// and writes the vertex in place (Eq. pbgn_update).
//
// Precision: element arithmetic is float32.  To keep it accurate for small
// strains, everything is formed relative to the rest state: H = F - I from
// displacement differences, J - 1 from the invariants of H, and R - I of the
// polar rotation from a quaternion whose vector part carries the rotation.
// Residual norms are accumulated in float64.
#include "pbng_internal.h"

#include <math.h>

namespace pbng {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }

// u_j - u_i from the stored pair: (hi_j - hi_i) + (lo_j - lo_i).
template <bool COMP>
__device__ __forceinline__ float3 disp_diff(const State& s, int j, float3 uh, float3 ul) {
    const float4 h = __ldg(s.hi + j);
    float3 d = make_float3(h.x - uh.x, h.y - uh.y, h.z - uh.z);
    if (COMP) {
        const float4 l = __ldg(s.lo + j);
        d.x += l.x - ul.x;
        d.y += l.y - ul.y;
        d.z += l.z - ul.z;
    }
    return d;
}

__device__ __forceinline__ float det3(float a, float b, float c, float d, float e, float f, float g,
                                      float h, float i) {
    return a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
}

// Rotation part of F = I + H for the corotated energy (Section "Constitutive
// Models", Eq. cor, with R the rotation of the polar decomposition in SO(3)).
//
// Method (Horn 1987, "Closed-form solution of absolute orientation using unit
// quaternions"; the polar use follows Higham & Noferini 2016): R(q) maximises
// tr(R^T F) over rotations, which is the SO(3) polar factor (the smallest
// singular value takes the sign of det F).  tr(R(q)^T F) = q^T N q for a
// traceless symmetric 4x4 N built linearly from F, so q is the eigenvector of
// N's largest eigenvalue.  Its characteristic polynomial is
//   p(t) = t^4 - 2|F|^2 t^2 - 8 det(F) t + |F|^4 - 4|cof F|^2,
// whose largest root is found by Newton from the upper bound sqrt(3)|F|
// (monotone, because p is real-rooted).  The eigenvector is a column of
// adj(N - t I), which is rank one; column 0 is used when it is well scaled
// (rotation angle up to about 120 degrees), else the column with the largest
// diagonal entry.  N - I_4-shifted is built from H, so the vector part of q,
// and with it R - I = 2w[v]x + 2[v]x^2, keep relative accuracy as H -> 0.
__device__ __forceinline__ void rotation_minus_identity(const float* H, float n2, float c2, float J,
                                                        float* RmI) {
    const float k0 = n2 * n2 - 4.0f * c2;
    float t = sqrtf(3.0f * n2);
    float dp = 1.0f;
#pragma unroll 1
    for (int it = 0; it < 12; ++it) {
        const float t2 = t * t;
        const float p = ((t2 - 2.0f * n2) * t - 8.0f * J) * t + k0;
        dp = (4.0f * t2 - 4.0f * n2) * t - 8.0f * J;
        const float d = p / dp;
        t -= d;
        if (!(fabsf(d) > 1e-7f * t)) break;
    }
    const float trH = H[0] + H[4] + H[8];
    const float m00 = (3.0f - t) + trH;
    const float m11 = (-1.0f - t) + (H[0] - H[4] - H[8]);
    const float m22 = (-1.0f - t) + (H[4] - H[0] - H[8]);
    const float m33 = (-1.0f - t) + (H[8] - H[0] - H[4]);
    const float m01 = H[7] - H[5], m02 = H[2] - H[6], m03 = H[3] - H[1];
    const float m12 = H[1] + H[3], m13 = H[2] + H[6], m23 = H[5] + H[7];
    // Column 0 of adj(M): (+min00, -min01, +min02, -min03).
    float q0 = det3(m11, m12, m13, m12, m22, m23, m13, m23, m33);
    float q1 = -det3(m01, m12, m13, m02, m22, m23, m03, m23, m33);
    float q2 = det3(m01, m11, m13, m02, m12, m23, m03, m13, m33);
    float q3 = -det3(m01, m11, m12, m02, m12, m22, m03, m13, m23);
    // adj(M) = -p'(t) q q^T, so q_0^2 = -adj_00 / p'(t).
    if (!(-q0 > 0.25f * dp)) {
        const float M[16] = {m00, m01, m02, m03, m01, m11, m12, m13,
                             m02, m12, m22, m23, m03, m13, m23, m33};
        float best = -q0;
        int kbest = 0;
        float colk[4];
        for (int k = 1; k < 4; ++k) {
            // diagonal entry adj_kk = det of M without row k and column k
            int r[3], n = 0;
            for (int i = 0; i < 4; ++i)
                if (i != k) r[n++] = i;
            const float dkk = det3(M[4 * r[0] + r[0]], M[4 * r[0] + r[1]], M[4 * r[0] + r[2]],
                                   M[4 * r[1] + r[0]], M[4 * r[1] + r[1]], M[4 * r[1] + r[2]],
                                   M[4 * r[2] + r[0]], M[4 * r[2] + r[1]], M[4 * r[2] + r[2]]);
            if (-dkk > best) { best = -dkk; kbest = k; }
        }
        if (kbest != 0) {
            for (int j = 0; j < 4; ++j) {
                // adj_jk = (-1)^{j+k} det(M without row k, column j)
                int rr[3], cc[3], nr = 0, nc = 0;
                for (int i = 0; i < 4; ++i) {
                    if (i != kbest) rr[nr++] = i;
                    if (i != j) cc[nc++] = i;
                }
                const float dm = det3(M[4 * rr[0] + cc[0]], M[4 * rr[0] + cc[1]], M[4 * rr[0] + cc[2]],
                                      M[4 * rr[1] + cc[0]], M[4 * rr[1] + cc[1]], M[4 * rr[1] + cc[2]],
                                      M[4 * rr[2] + cc[0]], M[4 * rr[2] + cc[1]], M[4 * rr[2] + cc[2]]);
                colk[j] = ((j + kbest) & 1) ? -dm : dm;
            }
            q0 = colk[0]; q1 = colk[1]; q2 = colk[2]; q3 = colk[3];
        }
    }
    const float qq = q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3;
    float w = 1.0f, x = 0.0f, y = 0.0f, z = 0.0f;
    if (qq > 1e-30f && isfinite(qq)) {
        const float inv = rsqrtf(qq);
        w = q0 * inv; x = q1 * inv; y = q2 * inv; z = q3 * inv;
    }
    // R - I = 2 w [v]x + 2 (v v^T - |v|^2 I), v = (x, y, z).
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

// Contribution of one incident tetrahedron (record s) to the force r and
// modified Hessian A (upper triangle a00 a01 a02 a11 a12 a22) of vertex i:
//   r -= V P(F) g_i,  P = 2 mu (F - R) + lambda (J - 1) cof F
//   A += V (2 mu |g_i|^2 I + lambda w w^T),  w = cof(F) g_i
// with F = I + sum_{j != i} (u_j - u_i) g_j^T and g_i = -(g_j1 + g_j2 + g_j3).
template <bool COMP, bool NEED_A>
__device__ __forceinline__ void element_term(const DeviceMesh& m, const State& s, int rec, float3 uh,
                                             float3 ul, float* r, float* A) {
    const float4 ra = __ldcs(m.rec_a + rec);
    const float4 rb = __ldcs(m.rec_b + rec);
    const float4 rc = __ldcs(m.rec_c + rec);
    const float2 rd = __ldcs(m.rec_d + rec);
    const float a = ra.w, b = rb.w;
    const float3 d1 = disp_diff<COMP>(s, __float_as_int(ra.x), uh, ul);
    const float3 d2 = disp_diff<COMP>(s, __float_as_int(ra.y), uh, ul);
    const float3 d3 = disp_diff<COMP>(s, __float_as_int(ra.z), uh, ul);
    const float g1[3] = {rb.x, rb.y, rb.z}, g2[3] = {rc.x, rc.y, rc.z}, g3[3] = {rc.w, rd.x, rd.y};
    const float dd1[3] = {d1.x, d1.y, d1.z}, dd2[3] = {d2.x, d2.y, d2.z}, dd3[3] = {d3.x, d3.y, d3.z};
    float H[9];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) H[3 * p + q] = dd1[p] * g1[q] + dd2[p] * g2[q] + dd3[p] * g3[q];
    const float gi[3] = {-(g1[0] + g2[0] + g3[0]), -(g1[1] + g2[1] + g3[1]), -(g1[2] + g2[2] + g3[2])};

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
    const float Jm1 = (H[0] + H[4] + H[8]) +
                      (H[0] * H[4] - H[1] * H[3] + H[0] * H[8] - H[2] * H[6] + H[4] * H[8] - H[5] * H[7]) +
                      det3(H[0], H[1], H[2], H[3], H[4], H[5], H[6], H[7], H[8]);
    float n2 = 0.0f, c2 = 0.0f;
    const float Fm[9] = {F0, F1, F2, F3, F4, F5, F6, F7, F8};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        n2 += Fm[k] * Fm[k];
        c2 += C[k] * C[k];
    }
    float RmI[9];
    rotation_minus_identity(H, n2, c2, 1.0f + Jm1, RmI);
    float w[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        w[p] = C[3 * p] * gi[0] + C[3 * p + 1] * gi[1] + C[3 * p + 2] * gi[2];
        const float fr = (H[3 * p] - RmI[3 * p]) * gi[0] + (H[3 * p + 1] - RmI[3 * p + 1]) * gi[1] +
                         (H[3 * p + 2] - RmI[3 * p + 2]) * gi[2];
        r[p] -= a * fr + b * Jm1 * w[p];
    }
    if (NEED_A) {
        const float ag = a * (gi[0] * gi[0] + gi[1] * gi[1] + gi[2] * gi[2]);
        A[0] += ag + b * w[0] * w[0];
        A[1] += b * w[0] * w[1];
        A[2] += b * w[0] * w[2];
        A[3] += ag + b * w[1] * w[1];
        A[4] += b * w[1] * w[2];
        A[5] += ag + b * w[2] * w[2];
    }
}

// Weak and contact terms of vertex v (internal free id) at displacement (uh + ul):
// springs r -= K (u - t_u), A += K I; plane contact with s = n.X - d + n.u < 0:
// r -= k s n, A += k n n^T.
template <bool COMP, bool NEED_A>
__device__ __forceinline__ void vertex_terms(const DeviceMesh& m, int v, float3 uh, float3 ul,
                                             float* r, float* A) {
    const float4 x0 = __ldg(m.aux0 + v);
    r[0] += x0.x;
    r[1] += x0.y;
    r[2] += x0.z;
    const float4 x1 = __ldg(m.aux1 + v);
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

// One vertex per W-lane group.  UPDATE: Eq. pbgn_dx / pbgn_update in place.
// Otherwise: write the residual of the vertex (lane 0 returns |r|^2 in rr).
template <int W, bool COMP, bool UPDATE>
__device__ __forceinline__ void vertex_group(const DeviceMesh& m, State s, int v, bool active,
                                             int lane, PassParams pp, int32_t* err, double* rr,
                                             float* r_out) {
    float3 uh = make_float3(0.f, 0.f, 0.f), ul = make_float3(0.f, 0.f, 0.f);
    int b0 = 0, b1 = 0;
    if (active) {
        uh = f3(s.hi[v]);
        if (COMP) ul = f3(s.lo[v]);
        b0 = __ldg(m.inc_off + v);
        b1 = __ldg(m.inc_off + v + 1);
    }
    float r[3] = {0.f, 0.f, 0.f};
    float A[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = b0 + lane; k < b1; k += W) element_term<COMP, UPDATE>(m, s, k, uh, ul, r, A);
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = group_sum<W>(r[k]);
    if (UPDATE) {
#pragma unroll
        for (int k = 0; k < 6; ++k) A[k] = group_sum<W>(A[k]);
    }
    if (!active || lane != 0) return;
    vertex_terms<COMP, UPDATE>(m, v, uh, ul, r, A);
    if (!UPDATE) {
        *rr = (double)r[0] * r[0] + (double)r[1] * r[1] + (double)r[2] * r[2];
        if (r_out) {
            r_out[3 * v] = r[0];
            r_out[3 * v + 1] = r[1];
            r_out[3 * v + 2] = r[2];
        }
        return;
    }
    if (pp.skip_tol > 0.0f && r[0] * r[0] + r[1] * r[1] + r[2] * r[2] <= pp.skip_tol * pp.skip_tol) return;
    // Delta = A^{-1} r by the adjugate (A symmetric positive definite).
    const float c00 = A[3] * A[5] - A[4] * A[4];
    const float c01 = A[2] * A[4] - A[1] * A[5];
    const float c02 = A[1] * A[4] - A[2] * A[3];
    const float c11 = A[0] * A[5] - A[2] * A[2];
    const float c12 = A[1] * A[2] - A[0] * A[4];
    const float c22 = A[0] * A[3] - A[1] * A[1];
    const float det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(det > 0.0f) || !isfinite(det)) {
        atomicOr(err, kErrNonSPD);
        return;
    }
    const float sc = pp.step / det;
    const float dx = sc * (c00 * r[0] + c01 * r[1] + c02 * r[2]);
    const float dy = sc * (c01 * r[0] + c11 * r[1] + c12 * r[2]);
    const float dz = sc * (c02 * r[0] + c12 * r[1] + c22 * r[2]);
    if (!(isfinite(dx) && isfinite(dy) && isfinite(dz))) {
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

__device__ __forceinline__ const Segment* find_segment(const SegmentTable& t, int block) {
    int k = 0;
    while (k + 1 < t.count && block >= t.seg[k + 1].block_begin) ++k;
    return &t.seg[k];
}

template <bool COMP, bool UPDATE>
__device__ __forceinline__ void dispatch(const DeviceMesh& m, State s, const Segment* sg, PassParams pp,
                                         int32_t* err, double* rr, float* r_out) {
    const int tid = (blockIdx.x - sg->block_begin) * kBlock + threadIdx.x;
    const int W = sg->width;
    const int v = sg->v_begin + tid / W;
    const bool active = v < sg->v_end;
    const int lane = tid & (W - 1);
    switch (W) {
        case 4: vertex_group<4, COMP, UPDATE>(m, s, v, active, lane, pp, err, rr, r_out); break;
        case 8: vertex_group<8, COMP, UPDATE>(m, s, v, active, lane, pp, err, rr, r_out); break;
        case 16: vertex_group<16, COMP, UPDATE>(m, s, v, active, lane, pp, err, rr, r_out); break;
        default: vertex_group<32, COMP, UPDATE>(m, s, v, active, lane, pp, err, rr, r_out); break;
    }
}

template <bool COMP>
__global__ void __launch_bounds__(kBlock) colour_pass_kernel(const DeviceMesh m, State s,
                                                             const SegmentTable t, PassParams pp,
                                                             int32_t* err) {
    const Segment* sg = find_segment(t, blockIdx.x);
    dispatch<COMP, true>(m, s, sg, pp, err, nullptr, nullptr);
}

// Residual of every free vertex (colour independent, no writes to the
// iterate); FP64 sums of |r_i|^2: one partial per block, or per component.
template <bool COMP>
__global__ void __launch_bounds__(kBlock) residual_kernel(const DeviceMesh m, State s,
                                                          const SegmentTable t, double* partial,
                                                          double* comp_sq, float* r_out) {
    const Segment* sg = find_segment(t, blockIdx.x);
    double rr = 0.0;
    dispatch<COMP, false>(m, s, sg, PassParams{1.f, 0.f}, nullptr, &rr, r_out);
    if (comp_sq) {
        const int tid = (blockIdx.x - sg->block_begin) * kBlock + threadIdx.x;
        const int v = sg->v_begin + tid / sg->width;
        if (rr != 0.0 && v < sg->v_end) atomicAdd(comp_sq + m.comp[v], rr);
        return;
    }
    // Block sum in a fixed order (warp shuffles, then shared memory).
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rr += __shfl_xor_sync(kFull, rr, off);
    __shared__ double ws[kBlock / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = rr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) tot += ws[k];
        partial[blockIdx.x] = tot;
    }
}

__global__ void reduce_kernel(const double* partial, int n, double* out) {
    __shared__ double sh[1024];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partial[k];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// Section "Acceleration Techniques", applied after a whole sweep:
//   x^{l+1} = w (g (x_P - x^l) + x^l - x^{l-1}) + x^{l-1}
// (Chebyshev: w = omega_{l+1}, g = gamma; SOR as printed: w = omega, g = 1).
// cur holds x_P on entry; p1 = x^l, p2 = x^{l-1}.  Writes x^{l+1} to cur and
// to p2 (the caller then swaps p1 and p2).
template <bool COMP>
__global__ void accel_kernel(int n, State cur, State p1, State p2, float w, float g) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    float4 xh = cur.hi[v], ah = p1.hi[v], bh = p2.hi[v];
    float4 xl = make_float4(0.f, 0.f, 0.f, 0.f), al = xl, bl = xl;
    if (COMP) { xl = cur.lo[v]; al = p1.lo[v]; bl = p2.lo[v]; }
    float o[3][2];
    const float X[3] = {xh.x, xh.y, xh.z}, XL[3] = {xl.x, xl.y, xl.z};
    const float Aa[3] = {ah.x, ah.y, ah.z}, AL[3] = {al.x, al.y, al.z};
    const float B[3] = {bh.x, bh.y, bh.z}, BL[3] = {bl.x, bl.y, bl.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float dP = X[k] - Aa[k], dD = Aa[k] - B[k];
        if (COMP) { dP += XL[k] - AL[k]; dD += AL[k] - BL[k]; }
        const float inc = w * (g * dP + dD);
        float hi = B[k], lo = BL[k];
        if (COMP) pair_add(hi, lo, inc);
        else hi += inc;
        o[k][0] = hi;
        o[k][1] = lo;
    }
    const float4 nh = make_float4(o[0][0], o[1][0], o[2][0], 0.f);
    cur.hi[v] = nh;
    p2.hi[v] = nh;
    if (COMP) {
        const float4 nl = make_float4(o[0][1], o[1][1], o[2][1], 0.f);
        cur.lo[v] = nl;
        p2.lo[v] = nl;
    }
}

// Caller layout -> internal state: free vertices take the caller's u, clamped
// ones their stored target displacement.
__global__ void load_kernel(int nv, int nfree, const float* u, const int32_t* perm,
                            const float4* dir_hi, const float4* dir_lo, State s) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    if (v < nfree) {
        const int o = perm[v];
        s.hi[v] = make_float4(u[3 * o], u[3 * o + 1], u[3 * o + 2], 0.f);
        s.lo[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        s.hi[v] = dir_hi[v - nfree];
        s.lo[v] = dir_lo[v - nfree];
    }
}

__global__ void store_kernel(int nv, const int32_t* perm, State s, float* u) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const float4 h = s.hi[v], l = s.lo[v];
    const int o = perm[v];
    u[3 * o] = h.x + l.x;
    u[3 * o + 1] = h.y + l.y;
    u[3 * o + 2] = h.z + l.z;
}

__global__ void copy_state_kernel(int n, State a, State b) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    b.hi[v] = a.hi[v];
    b.lo[v] = a.lo[v];
}

inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

}  // namespace

cudaError_t launch_colour_pass(const DeviceMesh& m, State s, const SegmentTable& t, PassParams p,
                               bool compensated, int32_t* err, cudaStream_t st) {
    if (t.total_blocks <= 0) return cudaSuccess;
    if (compensated) colour_pass_kernel<true><<<t.total_blocks, kBlock, 0, st>>>(m, s, t, p, err);
    else colour_pass_kernel<false><<<t.total_blocks, kBlock, 0, st>>>(m, s, t, p, err);
    return cudaGetLastError();
}

cudaError_t launch_residual(const DeviceMesh& m, State s, const SegmentTable& t, bool compensated,
                            double* block_partial, double* comp_sq, int32_t ncomp, float* r_out,
                            cudaStream_t st) {
    (void)ncomp;  // comp_sq is zeroed by the caller once per residual evaluation
    if (t.total_blocks <= 0) return cudaSuccess;
    if (compensated)
        residual_kernel<true><<<t.total_blocks, kBlock, 0, st>>>(m, s, t, block_partial, comp_sq, r_out);
    else
        residual_kernel<false><<<t.total_blocks, kBlock, 0, st>>>(m, s, t, block_partial, comp_sq, r_out);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double* partial, int32_t n, double* out, cudaStream_t st) {
    reduce_kernel<<<1, 1024, 0, st>>>(partial, n, out);
    return cudaGetLastError();
}

cudaError_t launch_accel(int32_t nfree, State cur, State p1, State p2, float w, float g,
                         bool compensated, cudaStream_t st) {
    if (nfree <= 0) return cudaSuccess;
    if (compensated) accel_kernel<true><<<blocks_for(nfree, 256), 256, 0, st>>>(nfree, cur, p1, p2, w, g);
    else accel_kernel<false><<<blocks_for(nfree, 256), 256, 0, st>>>(nfree, cur, p1, p2, w, g);
    return cudaGetLastError();
}

cudaError_t launch_load(int32_t nv, int32_t nfree, const float* u_user, const int32_t* perm,
                        const float4* dir_hi, const float4* dir_lo, State s, cudaStream_t st) {
    load_kernel<<<blocks_for(nv, 256), 256, 0, st>>>(nv, nfree, u_user, perm, dir_hi, dir_lo, s);
    return cudaGetLastError();
}

cudaError_t launch_store(int32_t nv, const int32_t* perm, State s, float* u_user, cudaStream_t st) {
    store_kernel<<<blocks_for(nv, 256), 256, 0, st>>>(nv, perm, s, u_user);
    return cudaGetLastError();
}

cudaError_t launch_copy_state(int32_t n, State src, State dst, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    copy_state_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}

}  // namespace pbng

// ---------------------------------------------------------------------------
// Fixed scratch for the allocation-free residual (pbng_residual_noalloc).
// One array per GPU that loads the library, kept until the process exits.
#include <mutex>

namespace pbng {
namespace {

constexpr int kNoAllocScratchDoubles = 1 << 16;  // 65,536 doubles = 512 KiB
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_noalloc_addr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

}  // namespace

int noalloc_scratch_capacity() { return kNoAllocScratchDoubles; }

// Device address of the scratch array on `device`, which must be current.
// The host-side name g_noalloc_scratch is only a stand-in; the address is
// looked up once per device with cudaGetSymbolAddress and cached.
cudaError_t noalloc_scratch(int device, double** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[device] = static_cast<double*>(p);
    }
    *out = g_noalloc_addr[device];
    return cudaSuccess;
}

}  // namespace pbng
