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
// Residuals sum each vertex's element terms, its vertex terms and the norms
// in float64.
#include "pbng_element.cuh"
#include "pbng_internal.h"
#include "pbng_launch.cuh"

#include <math.h>

namespace pbng {
namespace {

using el::kFull;
using el::f3;

// One vertex per W-lane group, direct loads from global memory (the path
// for small launches and for vertices with more than 256 incident tets).
// UPDATE: Eq. pbgn_dx / pbgn_update in place.  Otherwise the residual of the
// vertex (lane 0 returns |r|^2 in rr).
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
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = b0 + lane; k < b1; k += W) {
        const float4 ra = __ldcs(m.rec_a + k);
        const float4 rb = __ldcs(m.rec_b + k);
        const float4 rc = __ldcs(m.rec_c + k);
        const float2 rd = __ldcs(m.rec_d + k);
        const int j1 = __float_as_int(ra.x), j2 = __float_as_int(ra.y), j3 = __float_as_int(ra.z);
        const float3 d1 = el::pair_diff<COMP>(__ldg(s.hi + j1), COMP ? __ldg(s.lo + j1) : zero4, uh, ul);
        const float3 d2 = el::pair_diff<COMP>(__ldg(s.hi + j2), COMP ? __ldg(s.lo + j2) : zero4, uh, ul);
        const float3 d3 = el::pair_diff<COMP>(__ldg(s.hi + j3), COMP ? __ldg(s.lo + j3) : zero4, uh, ul);
        el::element_math<UPDATE>(pp.model, make_float3(rb.x, rb.y, rb.z), make_float3(rc.x, rc.y, rc.z),
                                 make_float3(rc.w, rd.x, rd.y), ra.w, rb.w, d1, d2, d3, r, A);
    }
    if (!UPDATE) {
        // residual: the W-lane sum of the float32 element terms and the
        // vertex terms in float-float
        ff::F2 rf[3] = {ff::mk(r[0]), ff::mk(r[1]), ff::mk(r[2])};
#pragma unroll
        for (int k = 0; k < 3; ++k) rf[k] = el::group_sum_ff<W>(rf[k]);
        if (!active || lane != 0) return;
        el::vertex_terms_ff<false>(m, v, __ldg(m.aux0 + v), __ldg(m.aux1 + v), uh, ul, rf, nullptr);
        el::weak_terms_ff<COMP, false>(m, s, v, rf, nullptr);
        *rr = el::norm2_ff(rf);
        if (r_out) {
            r_out[3 * v] = rf[0].h + rf[0].l;
            r_out[3 * v + 1] = rf[1].h + rf[1].l;
            r_out[3 * v + 2] = rf[2].h + rf[2].l;
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = el::group_sum<W>(r[k]);
#pragma unroll
    for (int k = 0; k < 6; ++k) A[k] = el::group_sum<W>(A[k]);
    if (!active || lane != 0) return;
    el::vertex_terms<COMP, UPDATE>(m, __ldg(m.aux0 + v), __ldg(m.aux1 + v), uh, ul, r, A);
    el::weak_terms<COMP, UPDATE>(m, s, v, r, A);
    if (m.comp_active && !m.comp_active[m.comp[v]]) return;  // frozen (converged) component
    el::solve_and_write<COMP>(s, v, uh, ul, r, A, pp, err);
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
    pdl_release();
    pdl_wait();
    const Segment* sg = find_segment(t, blockIdx.x);
    dispatch<COMP, true>(m, s, sg, pp, err, nullptr, nullptr);
}

// Residual of every free vertex (colour independent, no writes to the
// iterate); FP64 sums of |r_i|^2: one partial per block, or per component.
template <bool COMP>
__global__ void __launch_bounds__(kBlock) residual_kernel(const DeviceMesh m, State s,
                                                          const SegmentTable t, double* partial,
                                                          double* comp_sq, float* r_out, int model) {
    pdl_release();
    pdl_wait();
    const Segment* sg = find_segment(t, blockIdx.x);
    double rr = 0.0;
    dispatch<COMP, false>(m, s, sg, PassParams{1.f, 0.f, model}, nullptr, &rr, r_out);
    if (comp_sq) {
        const int tid = (blockIdx.x - sg->block_begin) * kBlock + threadIdx.x;
        const int v = sg->v_begin + tid / sg->width;
        if (v < sg->v_end && (tid & (sg->width - 1)) == 0) {
            if (m.vsq) m.vsq[v] = rr;  // summed per component in a fixed order afterwards
            else if (rr != 0.0) atomicAdd(comp_sq + m.comp[v], rr);
        }
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
    pdl_release();
    pdl_wait();
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

// Per-component sums of the vertices' |r|^2 in a fixed order, so that a
// batch's residuals (and its per-mesh stopping decisions) are the same bits
// on every run: one block per component sums vsq over its vertex list
// (internal ids) with a fixed thread-to-entry assignment and tree.
__global__ void __launch_bounds__(256) comp_reduce_kernel(const int32_t* __restrict__ off,
                                                          const int32_t* __restrict__ list,
                                                          const double* __restrict__ vsq, double* out) {
    pdl_release();
    pdl_wait();
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int k = off[c] + threadIdx.x; k < off[c + 1]; k += blockDim.x) acc += vsq[list[k]];
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
}

// Section "Acceleration Techniques", applied after a whole sweep:
//   x^{l+1} = w (g (x_P - x^l) + x^l - x^{l-1}) + x^{l-1}
// (Chebyshev: w = omega_{l+1}, g = gamma; SOR as printed: w = omega, g = 1).
// cur holds x_P on entry; p1 = x^l, p2 = x^{l-1}; (w, g) is read from device
// memory so a captured graph serves every sweep.  Writes x^{l+1} to cur and
// to p2 (the caller then swaps p1 and p2).
template <bool COMP>
__global__ void accel_kernel(int n, State cur, State p1, State p2, const float2* __restrict__ wg,
                             const int32_t* __restrict__ comp, const int32_t* __restrict__ active) {
    pdl_release();
    pdl_wait();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (active && !active[comp[v]]) return;  // frozen (converged) component
    const float w = wg->x, g = wg->y;
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
        if (COMP) el::pair_add(hi, lo, inc);
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

thread_local bool g_pdl = false;

}  // namespace

void set_pdl(bool on) { g_pdl = on; }
bool pdl_enabled() { return g_pdl; }

cudaError_t launch_colour_pass(const DeviceMesh& m, State s, const SegmentTable& t, PassParams p,
                               bool compensated, int32_t* err, cudaStream_t st) {
    if (t.total_blocks <= 0) return cudaSuccess;
    if (compensated) return launch_kernel(colour_pass_kernel<true>, t.total_blocks, kBlock, 0, st, m, s, t, p, err);
    return launch_kernel(colour_pass_kernel<false>, t.total_blocks, kBlock, 0, st, m, s, t, p, err);
}

cudaError_t launch_residual(const DeviceMesh& m, State s, const SegmentTable& t, bool compensated,
                            double* block_partial, double* comp_sq, int32_t ncomp, float* r_out, int model,
                            cudaStream_t st) {
    (void)ncomp;  // comp_sq is zeroed by the caller once per residual evaluation
    if (t.total_blocks <= 0) return cudaSuccess;
    if (compensated)
        return launch_kernel(residual_kernel<true>, t.total_blocks, kBlock, 0, st, m, s, t, block_partial, comp_sq,
                             r_out, model);
    return launch_kernel(residual_kernel<false>, t.total_blocks, kBlock, 0, st, m, s, t, block_partial, comp_sq,
                         r_out, model);
}

cudaError_t launch_reduce(const double* partial, int32_t n, double* out, cudaStream_t st) {
    return launch_kernel(reduce_kernel, 1, 1024, 0, st, partial, (int)n, out);
}

cudaError_t launch_comp_reduce(int32_t ncomp, const int32_t* off, const int32_t* list, const double* vsq,
                               double* out, cudaStream_t st) {
    if (ncomp <= 0) return cudaSuccess;
    return launch_kernel(comp_reduce_kernel, ncomp, 256, 0, st, off, list, vsq, out);
}

cudaError_t launch_accel(int32_t nfree, State cur, State p1, State p2, const float2* wg,
                         const int32_t* comp, const int32_t* comp_active, bool compensated, cudaStream_t st) {
    if (nfree <= 0) return cudaSuccess;
    if (compensated)
        return launch_kernel(accel_kernel<true>, blocks_for(nfree, 256), 256, 0, st, (int)nfree, cur, p1, p2, wg, comp,
                             comp_active);
    return launch_kernel(accel_kernel<false>, blocks_for(nfree, 256), 256, 0, st, (int)nfree, cur, p1, p2, wg, comp,
                         comp_active);
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

__global__ void inertia_kernel(int nv, int nfree, const int32_t* __restrict__ perm, float* u, float* u_prev,
                               const float4* __restrict__ base0, const float4* __restrict__ base1,
                               const float* __restrict__ k, float4* aux0, float4* aux1) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int o = perm[v];
    const float un[3] = {u[3 * o], u[3 * o + 1], u[3 * o + 2]};
    if (v < nfree) {
        const float4 b0 = base0[v], b1 = base1[v];
        const float kv = k[v], K = b0.w + kv;
        float t[3], g[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float uhat = 2.0f * un[a] - u_prev[3 * o + a];
            const float ts = (&b1.x)[a], fe = (&b0.x)[a];
            t[a] = K > 0.0f ? __fdividef(b0.w * ts + kv * uhat, K) : ts;
            g[a] = kv > 0.0f ? uhat + __fdividef(fe, kv) : un[a];
        }
        aux0[v] = make_float4(b0.x, b0.y, b0.z, K);
        aux1[v] = make_float4(t[0], t[1], t[2], b1.w);
#pragma unroll
        for (int a = 0; a < 3; ++a) u[3 * o + a] = g[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) u_prev[3 * o + a] = un[a];
}

cudaError_t launch_inertia(int32_t nv, int32_t nfree, const int32_t* perm, float* u, float* u_prev,
                           const float4* base0, const float4* base1, const float* k, float4* aux0, float4* aux1,
                           cudaStream_t st) {
    if (nv <= 0) return cudaSuccess;
    inertia_kernel<<<blocks_for(nv, 256), 256, 0, st>>>(nv, nfree, perm, u, u_prev, base0, base1, k, aux0, aux1);
    return cudaGetLastError();
}

cudaError_t launch_copy_state(int32_t n, State src, State dst, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    copy_state_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}

// FP32 FMA throughput probe (the roofline denominator of float32 element
// arithmetic): every thread runs kFmaChains independent FMA chains, enough
// to cover the FMA pipe's latency at full occupancy; one FMA = 2 flops.
constexpr int kFmaChains = 8;

__global__ void __launch_bounds__(256) fma_peak_kernel(float* out, int iters, float a, float b) {
    float x[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
    }
    float sum = 0.0f;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) sum += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = sum;  // keeps the chains live
}

cudaError_t fma_peak(cudaStream_t st, float* out, int blocks, int iters, cudaEvent_t e0, cudaEvent_t e1,
                     double* flops) {
    cudaError_t e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        fma_peak_kernel<<<blocks, 256, 0, st>>>(out, iters, 0.999999f, 1e-7f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    *flops = 2.0 * kFmaChains * (double)iters * (double)blocks * 256.0;
    return e;
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
