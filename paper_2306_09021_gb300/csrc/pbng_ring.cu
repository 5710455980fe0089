// Ring-layout colour passes and residuals for sm_103a.
//
// Layout: every free vertex of a colour owns W consecutive lanes of a
// 32-lane work item (W = 4, 8, 16 or 32), one W-lane group per vertex; its
// lanes hold the ids of its 1-ring vertices (the distinct vertices it shares
// a tet with) and records of its incident tets: dN/dX of the other three
// vertices, 2 mu V, lambda V, and the positions of those vertices in the
// item's 1-ring slots as bytes.
//   * Float32 passes and residuals (pair_kernel) read pair items (PairRec,
//     PairIds): two tets and two 1-ring vertices per lane, W the smallest
//     power of two holding half of each, and the element terms of both tets
//     in packed f32x2 arithmetic (pbng_pair.cuh).
//   * Extended-precision ones (ext_kernel) read ring items (RingBlock and
//     its low words RingLoBlock): one tet and one 1-ring vertex per lane,
//     float-float element forces (pbng_ff.cuh).
//
// Each warp is persistent and runs its own pipeline, with no block-wide
// barrier anywhere:
//   * lane 0 fetches an item's ids and records with TMA 1D bulk copies
//     (cp.async.bulk ... mbarrier::complete_tx) ahead of their use;
//   * once the ids land, every lane gathers the displacement pairs of its
//     1-ring vertices (and the item's own vertices and aux data) with
//     cp.async one item ahead, so each neighbour is read once per vertex
//     update, not once per incident tet;
//   * the compute forms u_j - u_i once per 1-ring vertex, hands each tet the
//     three it needs (shared memory for pair items, warp shuffles for ring
//     items), evaluates the element terms, sums the W lanes and adds the
//     vertex terms; in the float32 passes the group's first lane queues the
//     vertex's force and Hessian;
//   * when the warp's queue is nearly full (and at the end) all 32 lanes
//     solve and write one queued vertex each (Eq. pbgn_dx, Eq. pbgn_update),
//     instead of one lane per W-lane group solving while the others idle.
// Everything gathered by a pass belongs to other colours or to the item's own
// vertices, which only their own group writes; the vertices of one colour
// share no tet, so deferring their writes to the end of a queue changes
// nothing that another update of the same pass reads.
#include "pbng_async.cuh"
#include "pbng_element.cuh"
#include "pbng_ff.cuh"
#include "pbng_internal.h"
#include "pbng_launch.cuh"
#include "pbng_pair.cuh"

#include <stdint.h>

namespace pbng {
namespace {

using el::f3;
using el::kFull;
using namespace async;

constexpr int kWarps = kBlock / 32;
// 2 CTAs of 8 warps per SM: the packed element terms of two tets per lane
// take most of 128 registers, and the per-warp stages below half of an SM's
// shared memory.
constexpr int kCtasPerSm = 2;
constexpr int kGatStages = 2;
constexpr int kItemVerts = kRingLanes / 4;
constexpr int kQueue = 32;   // deferred vertex updates per warp

static_assert(kRingLanes == 32, "one record block per 32-lane item");

template <int NR>
struct __align__(16) GatStageT {
    float4 nh[NR];           // 1-ring displacement hi (pair items: u_j - u_i once formed)
    float4 nl[NR];           // 1-ring displacement lo
    float4 oh[kItemVerts];   // own vertex hi
    float4 ol[kItemVerts];   // own vertex lo
    float4 a0[kItemVerts];   // aux0 (f_ext, K), residual and extended passes only
    float4 a1[kItemVerts];   // aux1 (spring target, n.X - d), residual and extended passes only
};

// Force r (3) and modified Hessian A (6, upper triangle) of queued vertices,
// structure of arrays so the flush reads without bank conflicts; rows are
// padded to kQueue + 1 words so that the nine sums of one vertex, written
// by different lanes of its group, fall in nine different banks.  v = -1
// marks a frozen vertex that is not written.
struct __align__(16) UpdQueue {
    float val[9][kQueue + 1];
    int32_t v[kQueue];
};

// Extended passes: three stages of ring records (items requested two ahead)
// and of their low words, gathered with the 1-ring one item ahead.
constexpr int kExtStages = 3;
struct __align__(16) LoStage {
    float4 la[kRingLanes];
    float4 lb[kRingLanes];
    float4 lc[kRingLanes];
};
struct __align__(16) WarpSmemExt {
    RingBlock rec[kExtStages];
    GatStageT<kRingLanes> gat[kGatStages];
    LoStage lo[kGatStages];
    Item desc[kExtStages];
    unsigned long long bar[kExtStages];
};

// Float32 passes: the ids of an item are needed one item before its records
// (to gather its 1-ring), so they travel in their own bulk copies, two items
// ahead, and the records one item ahead.
constexpr int kIdStages = 3;
constexpr int kRecStages = 2;
static_assert(kIdStages == 3 && kRecStages == 2 && kGatStages == 2, "the pair pipeline advances its stages by hand");
struct __align__(16) WarpSmemPair {
    PairRec rec[kRecStages];
    PairIds ids[kIdStages];
    GatStageT<2 * kRingLanes> gat[kGatStages];
    UpdQueue q;
    Item desc[kIdStages];
    unsigned long long id_bar[kIdStages];
    unsigned long long rec_bar[kRecStages];
};

static_assert(kCtasPerSm * (kWarps * sizeof(WarpSmemPair) + 1024) <= 228 * 1024,
              "the per-warp stages of kCtasPerSm CTAs exceed an SM's shared memory");
static_assert(kCtasPerSm * (kWarps * sizeof(WarpSmemExt) + 1024) <= 228 * 1024,
              "the per-warp stages of kCtasPerSm extended CTAs exceed an SM's shared memory");
static_assert(sizeof(PairRec) % 16 == 0 && sizeof(PairIds) % 16 == 0 && sizeof(RingBlock) % 16 == 0,
              "bulk copies move multiples of 16 bytes");

// Whether item `it`'s whole component is frozen (then nothing is fetched).
__device__ __forceinline__ int item_skipped(const DeviceMesh& m, const Item& it) {
    return (it.comp >= 0 && m.comp_active && !m.comp_active[it.comp]) ? 1 : 0;
}

// Lane 0: one bulk copy of `bytes` (0 when the item is skipped) plus
// `extra` expected bytes (the timeout test hook) onto barrier `bar`.
__device__ __forceinline__ void issue_copy(void* dst, const void* src, uint32_t bytes, unsigned long long* bar,
                                           uint32_t extra = 0u) {
    mbar_arrive_expect_tx(bar, bytes + extra);
    if (bytes) bulk_g2s(dst, src, bytes, bar);
}

// Extended passes, lane 0: request the records and 1-ring ids of item `it`
// into stage r.  `extra` bytes are expected beyond the copy (the timeout
// test hook).
__device__ __forceinline__ void ext_issue_records(const DeviceMesh& m, Item it, WarpSmemExt& S, int r,
                                                  uint32_t extra = 0u) {
    it.skip = item_skipped(m, it);
    S.desc[r] = it;
    issue_copy(&S.rec[r], m.ring + (it.slot0 >> 5), it.skip ? 0u : (uint32_t)sizeof(RingBlock), S.bar + r,
               it.skip ? 0u : extra);
}

// Extended passes, all lanes: gather the 1-ring displacements, own-vertex
// and aux data and record low words of the item in record stage r into
// gather stage g.
__device__ __forceinline__ void ext_issue_gathers(const DeviceMesh& m, const State& s, WarpSmemExt& S, int r, int g,
                                                  int lane) {
    const Item it = S.desc[r];
    if (it.skip) return;
    auto& G = S.gat[g];
    const int id = S.rec[r].id[lane];
    cp_async16(G.nh + lane, s.hi + id);
    cp_async16(G.nl + lane, s.lo + id);
    if (lane < it.nv) {
        const int v = it.v0 + lane;
        cp_async16(G.oh + lane, s.hi + v);
        cp_async16(G.ol + lane, s.lo + v);
        cp_async16(G.a0 + lane, m.aux0 + v);
        cp_async16(G.a1 + lane, m.aux1 + v);
    }
    const RingLoBlock& L = m.ring_lo[it.slot0 >> 5];
    cp_async16(S.lo[g].la + lane, L.la + lane);
    cp_async16(S.lo[g].lb + lane, L.lb + lane);
    cp_async16(S.lo[g].lc + lane, L.lc + lane);
}

// Float32 passes, all lanes: gather the displacement pairs of the lane's two
// 1-ring slots and the item's own vertices (AUX: and their aux data, for the
// residual) of the item in id stage r into gather stage g.
template <bool COMP, bool AUX>
__device__ __forceinline__ void pair_issue_gathers(const DeviceMesh& m, const State& s, WarpSmemPair& S, int r, int g,
                                                   int lane) {
    const Item it = S.desc[r];
    if (it.skip) return;
    auto& G = S.gat[g];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int id = S.ids[r].id[h][lane];
        cp_async16(G.nh + h * kRingLanes + lane, s.hi + id);
        if (COMP) cp_async16(G.nl + h * kRingLanes + lane, s.lo + id);
    }
    if (lane < it.nv) {
        const int v = it.v0 + lane;
        cp_async16(G.oh + lane, s.hi + v);
        if (COMP) cp_async16(G.ol + lane, s.lo + v);
        if (AUX) {
            cp_async16(G.a0 + lane, m.aux0 + v);
            cp_async16(G.a1 + lane, m.aux1 + v);
        }
    }
}

// Reduce-scatter of a lane's 9 values (r, then A's upper triangle) over its
// W-lane group: log2(W) steps with offsets W/2 .. 1.  A step on N values keeps
// the first ceil(N/2) (lane bit clear) or the rest, zero-padded (bit set), and
// adds the partner's copy of the kept half, so after the last step a lane
// holds finished sums: one for W = 32 and 16, two for W = 8, three for W = 4
// (a step on one value is a plain pairwise sum).  Compared with nine
// separate W-lane sums this takes 12 shuffles instead of 45 for W = 32.
template <int N>
__device__ __forceinline__ void halve(float* v, int off, bool hi) {
    constexpr int h = (N + 1) / 2;
#pragma unroll
    for (int k = 0; k < h; ++k) {
        const float lo_v = v[k];
        const float hi_v = (h + k < N) ? v[h + k] : 0.0f;
        const float keep = hi ? hi_v : lo_v;
        const float send = hi ? lo_v : hi_v;
        v[k] = keep + __shfl_xor_sync(kFull, send, off);
    }
}

template <int N, int OFF>
__device__ __forceinline__ void butterfly(float* v, int lane) {
    if constexpr (OFF > 0) {
        if constexpr (N == 1) {
            v[0] += __shfl_xor_sync(kFull, v[0], OFF);
        } else {
            halve<N>(v, OFF, (lane & OFF) != 0);
        }
        butterfly<(N == 1 ? 1 : (N + 1) / 2), OFF / 2>(v, lane);
    }
}

// Index (0..8) of the sum a lane holds in final slot k, or -1 for padding.
template <int N, int OFF>
__device__ __forceinline__ int butterfly_index(int lane, int k) {
    if constexpr (OFF == 0) {
        return k < N ? k : -1;
    } else if constexpr (N == 1) {
        return butterfly_index<1, OFF / 2>(lane, k);
    } else {
        constexpr int h = (N + 1) / 2;
        const int p = butterfly_index<h, OFF / 2>(lane, k);
        if (p < 0) return -1;
        const int q = ((lane & OFF) ? h : 0) + p;
        return q < N ? q : -1;
    }
}

// Final slots per lane, and whether a lane writes them (for W = 32 the last
// step is a plain sum, so lanes 2i and 2i + 1 hold the same value).
template <int W>
struct ButterflyShape {
    static constexpr int slots = W >= 16 ? 1 : (W == 8 ? 2 : 3);
    static constexpr int shift = W == 32 ? 0 : (W == 16 ? 4 : (W == 8 ? 8 : 16));
    static __device__ __forceinline__ bool writer(int lane) { return W == 32 ? (lane & 1) == 0 : true; }
};

// butterfly_index of every lane width for this lane, computed once per
// kernel: 4 bits per final slot (15 = padding) at ButterflyShape<W>::shift.
__device__ __forceinline__ uint32_t butterfly_table(int lane) {
    uint32_t t = (uint32_t)(butterfly_index<9, 16>(lane, 0) & 15);
    t |= (uint32_t)(butterfly_index<9, 8>(lane, 0) & 15) << 4;
#pragma unroll
    for (int k = 0; k < 2; ++k) t |= (uint32_t)(butterfly_index<9, 4>(lane, k) & 15) << (8 + 4 * k);
#pragma unroll
    for (int k = 0; k < 3; ++k) t |= (uint32_t)(butterfly_index<9, 2>(lane, k) & 15) << (16 + 4 * k);
    return t;
}

// A vertex's |r|^2: into the warp's partial (one component), the vertex's
// slot of m.vsq (several components, summed per component in a fixed order
// afterwards), or atomically into its component's sum (several components,
// no slots: the allocation-free residual).
__device__ __forceinline__ void store_sq(const DeviceMesh& m, int v, double q, double& rr, double* comp_sq) {
    if (!comp_sq) rr += q;
    else if (m.vsq) m.vsq[v] = q;
    else atomicAdd(comp_sq + m.comp[v], q);
}

// Extended precision: the element force of the lane's slot in float-float
// arithmetic from float-pair records and displacements (pbng_ff.cuh), its
// W-lane sum and the vertex terms in float-float too; the nodal Hessian,
// which only scales the step, stays float32.  UPDATE: the group's first lane
// solves and writes its vertex at once (Eq. pbgn_dx, Eq. pbgn_update).
// Otherwise: |r|^2 of the vertex.
// The W-lane sums of the extended pass for a lane width known at compile
// time (f in float-float; A, the update's Hessian, in float).
template <int W, bool UPDATE>
__device__ __forceinline__ void ext_group_sums(ff::F2* f, float* A) {
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = el::group_sum_ff<W>(f[k]);
    if (UPDATE) {
#pragma unroll
        for (int k = 0; k < 6; ++k) A[k] = el::group_sum<W>(A[k]);
    }
}

// The lane width W = it.w is a run-time value everywhere but in the W-lane
// sums: one copy of the long float-float element force per kernel instead
// of one per width keeps the kernel within the instruction cache.
template <bool UPDATE, int MODEL>
__device__ __forceinline__ void compute_item_ext(const DeviceMesh& m, State s, WarpSmemExt& S, const Item& it, int r,
                                                 int g, int lane, PassParams pp, int32_t* err, double& rr,
                                                 double* comp_sq) {
    const RingBlock& R = S.rec[r];
    const auto& G = S.gat[g];
    const int W = it.w;
    const int j = lane >> (__ffs(W) - 1);
    const bool active = j < it.nv;
    float3 uh = make_float3(0.f, 0.f, 0.f), ul = uh;
    // u_j - u_i as an exact float pair: (hi_j - hi_i) by TwoSum, plus the low words
    ff::F2 dv[3] = {ff::mk(0.f), ff::mk(0.f), ff::mk(0.f)};
    if (active) {
        uh = f3(G.oh[j]);
        ul = f3(G.ol[j]);
        const float4 hj = G.nh[lane], lj = G.nl[lane];
        dv[0] = ff::add(ff::two_sum(hj.x, -uh.x), ff::fadd(lj.x, -ul.x));
        dv[1] = ff::add(ff::two_sum(hj.y, -uh.y), ff::fadd(lj.y, -ul.y));
        dv[2] = ff::add(ff::two_sum(hj.z, -uh.z), ff::fadd(lj.z, -ul.z));
    }
    const float4 ra = R.ra[lane], rb = R.rb[lane], rc = R.rc[lane];
    const LoStage& L = S.lo[g];
    const float4 la = L.la[lane], lb = L.lb[lane], lc = L.lc[lane];
    const int loc = __float_as_int(rc.w);
    const int base = lane & ~(W - 1);
    const int src[3] = {base + (loc & 255), base + ((loc >> 8) & 255), base + ((loc >> 16) & 255)};
    ff::F2 d[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            d[k][c] = ff::mk(__shfl_sync(kFull, dv[c].h, src[k]), __shfl_sync(kFull, dv[c].l, src[k]));
    const ff::F2 gg[3][3] = {{ff::mk(ra.x, la.x), ff::mk(ra.y, la.y), ff::mk(ra.z, la.z)},
                             {ff::mk(rb.x, lb.x), ff::mk(rb.y, lb.y), ff::mk(rb.z, lb.z)},
                             {ff::mk(rc.x, lc.x), ff::mk(rc.y, lc.y), ff::mk(rc.z, lc.z)}};
    float A[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float q[4] = {1.f, 0.f, 0.f, 0.f};
    el::element_fp32_parts<UPDATE, MODEL == el::kCorotated>(
        f3(ra), f3(rb), f3(rc), ra.w, rb.w, make_float3(d[0][0].h, d[0][1].h, d[0][2].h),
        make_float3(d[1][0].h, d[1][1].h, d[1][2].h), make_float3(d[2][0].h, d[2][1].h, d[2][2].h), A, q);
    ff::F2 f[3];
    ff::element_force<MODEL>(gg, ff::mk(ra.w, la.w), ff::mk(rb.w, lb.w), d, q, f);
    switch (W) {  // warp-uniform
        case 4: ext_group_sums<4, UPDATE>(f, A); break;
        case 8: ext_group_sums<8, UPDATE>(f, A); break;
        case 16: ext_group_sums<16, UPDATE>(f, A); break;
        default: ext_group_sums<32, UPDATE>(f, A); break;
    }
    if (!active || (lane & (W - 1)) != 0) return;
    const int v = it.v0 + j;
    el::vertex_terms_ff<UPDATE>(m, v, G.a0[j], G.a1[j], uh, ul, f, A);
    el::weak_terms_ff<true, UPDATE>(m, s, v, f, A);
    if constexpr (UPDATE) {
        if (it.comp < 0 && m.comp_active && !m.comp_active[m.comp[v]]) return;  // frozen vertex of a mixed item
        const float rf[3] = {f[0].h + f[0].l, f[1].h + f[1].l, f[2].h + f[2].l};
        el::solve_and_write<true>(s, v, uh, ul, rf, A, pp, err);
    } else {
        if (m.fout_hi) {
            m.fout_hi[v] = make_float4(f[0].h, f[1].h, f[2].h, 0.f);
            m.fout_lo[v] = make_float4(f[0].l, f[1].l, f[2].l, 0.f);
        }
        store_sq(m, v, el::norm2_ff(f), rr, comp_sq);
    }
}

// Float32: the element terms of the lane's two tets (A = tet l, B = tet
// W + l of its group's vertex) in packed f32x2 arithmetic, their sum, the
// W-lane sums of the group.  Each lane first forms u_j - u_i of its two
// 1-ring slots in place in the gather stage; every tet then reads the three
// differences it needs from there.  UPDATE: the sums go straight into the
// warp's queue from the lanes that hold them; the vertex terms are added
// when the queue is flushed.  Otherwise: the element sums in float32, their
// W-lane sum and the vertex terms in float-float, and |r|^2 of the vertex.
template <int W, bool COMP, bool UPDATE, int MODEL>
__device__ __forceinline__ void compute_item_pair(const DeviceMesh& m, State s, WarpSmemPair& S, const Item& it, int r,
                                                  int g, int lane, uint32_t btab, int qn, double& rr,
                                                  double* comp_sq) {
    const PairRec& R = S.rec[r];
    auto& G = S.gat[g];
    const int j = lane / W;
    const bool active = j < it.nv;
    const float3 zero3 = make_float3(0.f, 0.f, 0.f);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float3 uh = zero3, ul = zero3;
    if (active) {
        uh = f3(G.oh[j]);
        if (COMP) ul = f3(G.ol[j]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = h * kRingLanes + lane;  // only this lane reads or writes slot k here
        float3 d = zero3;
        if (active) d = el::pair_diff<COMP>(G.nh[k], COMP ? G.nl[k] : zero4, uh, ul);
        G.nh[k] = make_float4(d.x, d.y, d.z, 0.f);
    }
    __syncwarp();
    float4 q[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = R.r[k][lane];
    // value k of the pair: (q[k/2].x, .y) for even k, (.z, .w) for odd k
    const float2 g1[3] = {make_float2(q[0].x, q[0].y), make_float2(q[0].z, q[0].w), make_float2(q[1].x, q[1].y)};
    const float2 g2[3] = {make_float2(q[1].z, q[1].w), make_float2(q[2].x, q[2].y), make_float2(q[2].z, q[2].w)};
    const float2 g3[3] = {make_float2(q[3].x, q[3].y), make_float2(q[3].z, q[3].w), make_float2(q[4].x, q[4].y)};
    const float2 a = make_float2(q[4].z, q[4].w), b = make_float2(q[5].x, q[5].y);
    const int locA = __float_as_int(q[5].z), locB = __float_as_int(q[5].w);
    const int base = lane & ~(W - 1);
    float2 dk[3][3];  // dk[k][c]: component c of u_jk - u_i, (tet A, tet B)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 dA = G.nh[base + ((locA >> (8 * k)) & 255)];
        const float4 dB = G.nh[base + ((locB >> (8 * k)) & 255)];
        dk[k][0] = make_float2(dA.x, dB.x);
        dk[k][1] = make_float2(dA.y, dB.y);
        dk[k][2] = make_float2(dA.z, dB.z);
    }
    float2 f2[3], A2[6];
    pk::element_math_pair<UPDATE, MODEL>(g1, g2, g3, a, b, dk[0], dk[1], dk[2], f2, A2);
    float rv[3], A[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) rv[k] = f2[k].x + f2[k].y;
    if constexpr (UPDATE) {
#pragma unroll
        for (int k = 0; k < 6; ++k) A[k] = A2[k].x + A2[k].y;
        float val[9] = {rv[0], rv[1], rv[2], A[0], A[1], A[2], A[3], A[4], A[5]};
        butterfly<9, W / 2>(val, lane);
        const int e = qn + j;
        if (active && ButterflyShape<W>::writer(lane)) {
#pragma unroll
            for (int k = 0; k < ButterflyShape<W>::slots; ++k) {
                const int idx = (int)((btab >> (ButterflyShape<W>::shift + 4 * k)) & 15u);
                if (idx < 9) S.q.val[idx][e] = val[k];
            }
        }
        if (!active || (lane & (W - 1)) != 0) return;
        const int v = it.v0 + j;
        // a frozen vertex of a mixed item is not written
        S.q.v[e] = (it.comp < 0 && m.comp_active && !m.comp_active[m.comp[v]]) ? -1 : v;
    } else {
        ff::F2 rf[3] = {ff::mk(rv[0]), ff::mk(rv[1]), ff::mk(rv[2])};
#pragma unroll
        for (int k = 0; k < 3; ++k) rf[k] = el::group_sum_ff<W>(rf[k]);
        if (!active || (lane & (W - 1)) != 0) return;
        const int v = it.v0 + j;
        el::vertex_terms_ff<false>(m, v, G.a0[j], G.a1[j], uh, COMP ? ul : zero3, rf, nullptr);
        el::weak_terms_ff<COMP, false>(m, s, v, rf, nullptr);
        store_sq(m, v, el::norm2_ff(rf), rr, comp_sq);
    }
}

// All lanes: solve and write the qn queued vertices, one per lane.  The own
// displacement is read again here; no other update of the pass writes it.
template <bool COMP>
__device__ __forceinline__ void flush_queue(const DeviceMesh& m, State s, const UpdQueue& Q, int qn, int lane,
                                            PassParams pp, int32_t* err) {
    __syncwarp();
    if (lane < qn) {
        const int v = Q.v[lane];
        if (v >= 0) {
            float rv[3], A[6];
#pragma unroll
            for (int k = 0; k < 3; ++k) rv[k] = Q.val[k][lane];
#pragma unroll
            for (int k = 0; k < 6; ++k) A[k] = Q.val[3 + k][lane];
            const float3 uh = f3(s.hi[v]);
            const float3 ul = COMP ? f3(s.lo[v]) : make_float3(0.f, 0.f, 0.f);
            el::vertex_terms<COMP, true>(m, m.aux0[v], m.aux1[v], uh, ul, rv, A);
            el::weak_terms<COMP, true>(m, s, v, rv, A);
            el::solve_and_write<COMP>(s, v, uh, ul, rv, A, pp, err);
        }
    }
    __syncwarp();
}

// Item order of a pass: strided (warp gw takes items gw, gw + nw, ...) or
// blocked (warp gw takes a contiguous run of ceil(nitems / nw) items).  The
// order only decides which warp updates which vertices of one colour; the
// updates of a colour are independent, so the iterate is the same.
__device__ __forceinline__ void item_range(int blocked, int nitems, int gw, int nw, int& n, int& first,
                                           int& stride) {
    if (blocked) {
        const int per = (nitems + nw - 1) / nw;
        first = gw * per;
        stride = 1;
        n = nitems - first < per ? nitems - first : per;
        if (n < 0) n = 0;
    } else {
        first = gw;
        stride = nw;
        n = gw < nitems ? (nitems - gw + nw - 1) / nw : 0;
    }
}

// The warp's FP64 residual partial (one per warp of the grid; idle warps
// write zero after the predecessor kernel).
__device__ __forceinline__ void write_partial(double rr, int n, int lane, int gw, double* partial) {
    if (n == 0) pdl_wait();  // idle warp: order its write after the predecessor
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rr += __shfl_xor_sync(kFull, rr, off);
    if (lane == 0) partial[gw] = rr;
}

// Extended-precision colour pass (UPDATE) or residual over ring items.
template <bool UPDATE, int MODEL>
__global__ void __launch_bounds__(kBlock, kCtasPerSm)
    ext_kernel(const DeviceMesh m, State s, const Item* __restrict__ items, int nitems, PassParams pp,
               int32_t* err, double* partial, double* comp_sq, int blocked) {
    constexpr int RS = kExtStages, RA = kExtStages - 1;  // items' records are requested RA ahead
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_release();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmemExt& S = reinterpret_cast<WarpSmemExt*>(smem)[warp];
    const int gw = (int)blockIdx.x * kWarps + warp, nw = (int)gridDim.x * kWarps;
    int n, first, stride;
    item_range(blocked, nitems, gw, nw, n, first, stride);
    double rr = 0.0;
    int issued = 0, waited = 0;  // items whose records were requested / awaited
    bool ok = true;
    Item next{};                 // lane 0: next item to request, loaded one item early
    if (n > 0) {
        if (lane == 0) {
            for (int i = 0; i < RS; ++i) mbar_init(S.bar + i, 1);
            fence_mbar_init();
            for (int i = 0; i < RA && i < n; ++i)
                ext_issue_records(m, items[first + i * stride], S, i, i == 0 ? (uint32_t)m.copy_shortfall : 0u);
            if (n > RA) next = items[first + RA * stride];
        }
        issued = n < RA ? n : RA;
        __syncwarp();
        // Records, items and component flags are written by no kernel; the
        // iterate read from here on is written by the previous kernel.
        pdl_wait();
        ok = mbar_wait(S.bar + 0, 0);
        waited = ok ? 1 : 0;  // a stage whose wait gave up is drained again on abort
        if (__any_sync(kFull, !ok)) goto abort;
        ext_issue_gathers(m, s, S, 0, 0, lane);
        cp_async_commit();
        for (int k = 0; k < n; ++k) {
            // Record stage (k + RA) % RS and gather stage (k+1)%2 were last
            // read by item k-1, finished before the previous __syncwarp.
            if (k + RA < n) {
                if (lane == 0) {
                    fence_proxy_async();
                    ext_issue_records(m, next, S, (k + RA) % RS);
                    if (k + RA + 1 < n) next = items[first + (k + RA + 1) * stride];
                }
                issued = k + RA + 1;
            }
            ok = true;
            if (k + 1 < n) {
                ok = mbar_wait(S.bar + (k + 1) % RS, ((k + 1) / RS) & 1);
                waited = ok ? k + 2 : k + 1;
                if (ok) ext_issue_gathers(m, s, S, (k + 1) % RS, (k + 1) % kGatStages, lane);
            }
            cp_async_commit();
            cp_async_wait<1>();  // this lane's gathers of item k have landed
            if (__any_sync(kFull, !ok)) goto abort;
            __syncwarp();        // ... and the other lanes'
            const Item it = S.desc[k % RS];
            const int r = k % RS, g = k % kGatStages;
            if (!it.skip) compute_item_ext<UPDATE, MODEL>(m, s, S, it, r, g, lane, pp, err, rr, comp_sq);  // warp-uniform
            __syncwarp();
        }
    }
    if (!UPDATE && partial) write_partial(rr, n, lane, gw, partial);
    return;

abort:
    // A record copy did not complete in time: report it, let the copies this
    // warp started finish (bounded), then leave.
    if (lane == 0) {
        atomicOr(err, kErrTimeout);
        for (int k = waited; k < issued; ++k) (void)mbar_wait(S.bar + k % RS, (k / RS) & 1);
        if (!UPDATE && partial) partial[gw] = 0.0;
    }
    cp_async_wait<0>();
    __syncwarp();
}

// Float32 passes, lane 0: request the ids of item `it` into id stage r
// (`extra` expected bytes beyond the copy: the timeout test hook) and
// record the item in desc[r].
__device__ __forceinline__ void pair_issue_ids(const DeviceMesh& m, Item it, WarpSmemPair& S, int r,
                                               uint32_t extra = 0u) {
    it.skip = item_skipped(m, it);
    S.desc[r] = it;
    issue_copy(&S.ids[r], m.pids + (it.slot0 >> 5), it.skip ? 0u : (uint32_t)sizeof(PairIds), S.id_bar + r,
               it.skip ? 0u : extra);
}

// Float32 passes, lane 0: request the records of the item in id stage r
// into record stage q.
__device__ __forceinline__ void pair_issue_rec(const DeviceMesh& m, WarpSmemPair& S, int r, int q) {
    const Item it = S.desc[r];
    issue_copy(&S.rec[q], m.prec + (it.slot0 >> 5), it.skip ? 0u : (uint32_t)sizeof(PairRec), S.rec_bar + q);
}

// Float32 colour pass (UPDATE) or residual over pair items.  Item k's ids
// are requested at iteration k - 2 and awaited at k - 1, where its gathers
// are issued; its records are requested at k - 1 and awaited at k.
template <bool COMP, bool UPDATE, int MODEL>
__global__ void __launch_bounds__(kBlock, kCtasPerSm)
    pair_kernel(const DeviceMesh m, State s, const Item* __restrict__ items, int nitems, PassParams pp,
                int32_t* err, double* partial, double* comp_sq, int blocked) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_release();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmemPair& S = reinterpret_cast<WarpSmemPair*>(smem)[warp];
    const int gw = (int)blockIdx.x * kWarps + warp, nw = (int)gridDim.x * kWarps;
    int n, first, stride;
    item_range(blocked, nitems, gw, nw, n, first, stride);
    double rr = 0.0;
    const uint32_t btab = UPDATE ? butterfly_table(lane) : 0u;
    int qn = 0;  // queued vertex updates (warp-uniform)
    // items whose ids / records were requested, and those awaited (a stage
    // whose wait gave up is drained again on abort)
    int id_issued = 0, id_waited = 0, rec_issued = 0, rec_waited = 0;
    bool ok = true;
    Item next{};  // lane 0: the next item whose ids are requested
    if (n > 0) {
        if (lane == 0) {
            for (int i = 0; i < kIdStages; ++i) mbar_init(S.id_bar + i, 1);
            for (int i = 0; i < kRecStages; ++i) mbar_init(S.rec_bar + i, 1);
            fence_mbar_init();
            for (int i = 0; i < 2 && i < n; ++i)
                pair_issue_ids(m, items[first + i * stride], S, i, i == 0 ? (uint32_t)m.copy_shortfall : 0u);
            pair_issue_rec(m, S, 0, 0);
            if (n > 2) next = items[first + 2 * stride];
        }
        id_issued = n < 2 ? n : 2;
        rec_issued = 1;
        __syncwarp();
        // Records, ids, items and component flags are written by no kernel;
        // the iterate read from here on is written by the previous kernel.
        pdl_wait();
        ok = mbar_wait(S.id_bar + 0, 0);
        id_waited = ok ? 1 : 0;
        if (__any_sync(kFull, !ok)) goto abort;
        pair_issue_gathers<COMP, !UPDATE>(m, s, S, 0, 0, lane);
        cp_async_commit();
        // stages and barrier parities, advanced each item: id stage of items
        // k, k + 1, k + 2 and the parity of item k + 1's; record and gather
        // stage of item k and the parity of its record barrier
        int i0 = 0, i1 = 1, i2 = 2, ph1 = 0, r0 = 0, rph = 0;
        for (int k = 0; k < n; ++k) {
            // Id stage i2 was last read by the gathers of item k - 1, record
            // stage 1 - r0 and gather stage 1 - r0 by the compute of item
            // k - 1, all finished before the previous __syncwarp.
            if (lane == 0) {
                fence_proxy_async();
                if (k + 2 < n) {
                    pair_issue_ids(m, next, S, i2);
                    if (k + 3 < n) next = items[first + (k + 3) * stride];
                }
                if (k + 1 < n) pair_issue_rec(m, S, i1, r0 ^ 1);
            }
            if (k + 2 < n) id_issued = k + 3;
            if (k + 1 < n) rec_issued = k + 2;
            ok = true;
            if (k + 1 < n) {
                ok = mbar_wait(S.id_bar + i1, ph1);
                id_waited = ok ? k + 2 : k + 1;
                if (ok) pair_issue_gathers<COMP, !UPDATE>(m, s, S, i1, r0 ^ 1, lane);
            }
            cp_async_commit();
            const bool rok = mbar_wait(S.rec_bar + r0, rph);
            rec_waited = rok ? k + 1 : k;
            cp_async_wait<1>();  // this lane's gathers of item k have landed
            if (__any_sync(kFull, !(ok && rok))) goto abort;
            __syncwarp();        // ... and the other lanes'
            const Item it = S.desc[i0];
            if (!it.skip) {  // uniform over the warp; the lane width too
                // pair widths are 4, 8 or 16: a ring colour's vertices have at
                // most 32 tets and 32 1-ring vertices (the layout checks it)
                switch (it.w) {
                    case 4: compute_item_pair<4, COMP, UPDATE, MODEL>(m, s, S, it, r0, r0, lane, btab, qn, rr, comp_sq); break;
                    case 8: compute_item_pair<8, COMP, UPDATE, MODEL>(m, s, S, it, r0, r0, lane, btab, qn, rr, comp_sq); break;
                    default: compute_item_pair<16, COMP, UPDATE, MODEL>(m, s, S, it, r0, r0, lane, btab, qn, rr, comp_sq); break;
                }
            }
            if (UPDATE) {
                if (!it.skip) qn += it.nv;
                if (qn > kQueue - kItemVerts || (k + 1 == n && qn > 0)) {
                    flush_queue<COMP>(m, s, S.q, qn, lane, pp, err);
                    qn = 0;
                }
            }
            __syncwarp();
            i0 = i1;
            i1 = i2;
            i2 = i2 == kIdStages - 1 ? 0 : i2 + 1;
            if (i1 == 0) ph1 ^= 1;
            r0 ^= 1;
            if (r0 == 0) rph ^= 1;
        }
    }
    if (!UPDATE && partial) write_partial(rr, n, lane, gw, partial);
    return;

abort:
    // An id or record copy did not complete in time: report it, let the
    // copies this warp started finish (bounded), then leave.
    if (lane == 0) {
        atomicOr(err, kErrTimeout);
        for (int k = id_waited; k < id_issued; ++k) (void)mbar_wait(S.id_bar + k % kIdStages, (k / kIdStages) & 1);
        for (int k = rec_waited; k < rec_issued; ++k)
            (void)mbar_wait(S.rec_bar + k % kRecStages, (k / kRecStages) & 1);
        if (!UPDATE && partial) partial[gw] = 0.0;
    }
    cp_async_wait<0>();
    __syncwarp();
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
        cached[dev] = nsm;
    }
    return cached[dev];
}

int ring_ctas(int nitems, int ctas_per_sm, int balanced = 0) {
    const int want = (nitems + kWarps - 1) / kWarps;
    const int cps = ctas_per_sm < 1 ? 1 : (ctas_per_sm > kCtasPerSm ? kCtasPerSm : ctas_per_sm);
    const int cap = cps * sm_count();
    int grid = want < cap ? want : cap;
    if (balanced && grid > 0) {
        // the same number of item rounds with the fewest warps
        const int rounds = (nitems + grid * kWarps - 1) / (grid * kWarps);
        const int warps = (nitems + rounds - 1) / rounds;
        grid = (warps + kWarps - 1) / kWarps;
    }
    return grid;
}

// grid_warps > 0: a grid of exactly that many warps (a multiple of kWarps;
// the residuals, whose partials are one per warp); else the schedule's.
template <bool COMP, bool UPDATE, bool EXT>
cudaError_t launch_impl(const DeviceMesh& m, State s, const Item* items, int nitems, PassParams pp,
                        int32_t* err, double* partial, double* comp_sq, RingSched sc, cudaStream_t st,
                        int grid_warps = 0) {
    if (nitems <= 0 && grid_warps <= 0) return cudaSuccess;
    const int grid = grid_warps > 0 ? grid_warps / kWarps : ring_ctas(nitems, sc.ctas_per_sm, sc.balanced);
    if constexpr (EXT) {
        const int bytes = kWarps * (int)sizeof(WarpSmemExt);  // attribute set by ring_prepare()
        if (pp.model == el::kNeoHookean)
            return launch_kernel(ext_kernel<UPDATE, el::kNeoHookean>, grid, kBlock, bytes, st, m, s, items, nitems,
                                 pp, err, partial, comp_sq, sc.blocked);
        if (pp.model == el::kStableNeoHookean)
            return launch_kernel(ext_kernel<UPDATE, el::kStableNeoHookean>, grid, kBlock, bytes, st, m, s, items,
                                 nitems, pp, err, partial, comp_sq, sc.blocked);
        return launch_kernel(ext_kernel<UPDATE, el::kCorotated>, grid, kBlock, bytes, st, m, s, items, nitems, pp,
                             err, partial, comp_sq, sc.blocked);
    } else {
        const int bytes = kWarps * (int)sizeof(WarpSmemPair);
        if (pp.model == el::kNeoHookean)
            return launch_kernel(pair_kernel<COMP, UPDATE, el::kNeoHookean>, grid, kBlock, bytes, st, m, s, items,
                                 nitems, pp, err, partial, comp_sq, sc.blocked);
        if (pp.model == el::kStableNeoHookean)
            return launch_kernel(pair_kernel<COMP, UPDATE, el::kStableNeoHookean>, grid, kBlock, bytes, st, m, s,
                                 items, nitems, pp, err, partial, comp_sq, sc.blocked);
        return launch_kernel(pair_kernel<COMP, UPDATE, el::kCorotated>, grid, kBlock, bytes, st, m, s, items, nitems,
                             pp, err, partial, comp_sq, sc.blocked);
    }
}

}  // namespace

int ring_warps(int nitems) { return nitems > 0 ? ring_ctas(nitems, kCtasPerSm) * kWarps : 0; }

int ring_max_ctas_per_sm() { return kCtasPerSm; }

cudaError_t ring_prepare() {
    // Two CTAs of 8 warps with their per-warp stages and queues need almost
    // all of an SM's shared memory: ask for the largest carveout.
    const int bytes = kWarps * (int)sizeof(WarpSmemPair), bytes_ext = kWarps * (int)sizeof(WarpSmemExt);
    const void* fns[18] = {
        (const void*)pair_kernel<true, true, 0>,  (const void*)pair_kernel<false, true, 0>,
        (const void*)pair_kernel<true, false, 0>, (const void*)pair_kernel<false, false, 0>,
        (const void*)pair_kernel<true, true, 1>,  (const void*)pair_kernel<false, true, 1>,
        (const void*)pair_kernel<true, false, 1>, (const void*)pair_kernel<false, false, 1>,
        (const void*)pair_kernel<true, true, 2>,  (const void*)pair_kernel<false, true, 2>,
        (const void*)pair_kernel<true, false, 2>, (const void*)pair_kernel<false, false, 2>,
        (const void*)ext_kernel<true, 0>,         (const void*)ext_kernel<false, 0>,
        (const void*)ext_kernel<true, 1>,         (const void*)ext_kernel<false, 1>,
        (const void*)ext_kernel<true, 2>,         (const void*)ext_kernel<false, 2>};
    for (int k = 0; k < 18; ++k) {
        const void* f = fns[k];
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, k < 12 ? bytes : bytes_ext);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_ring_pass(const DeviceMesh& m, State s, const Item* items, int nitems, PassParams p,
                             bool compensated, RingSched sc, int32_t* err, cudaStream_t st, bool extended) {
    if (extended) {
        if (!compensated || !m.ring_lo) return cudaErrorInvalidValue;
        return launch_impl<true, true, true>(m, s, items, nitems, p, err, nullptr, nullptr, sc, st);
    }
    if (compensated) return launch_impl<true, true, false>(m, s, items, nitems, p, err, nullptr, nullptr, sc, st);
    return launch_impl<false, true, false>(m, s, items, nitems, p, err, nullptr, nullptr, sc, st);
}

cudaError_t launch_ring_residual(const DeviceMesh& m, State s, const Item* items, int nitems,
                                 bool compensated, double* warp_partial, double* comp_sq, int model, int32_t* err,
                                 cudaStream_t st, bool extended, int grid_warps) {
    const PassParams pp{1.f, 0.f, model};
    const RingSched sc{kCtasPerSm, 0, 0};
    double* part = comp_sq ? nullptr : warp_partial;
    if (grid_warps <= 0 || grid_warps % kWarps) return cudaErrorInvalidValue;
    if (extended) {
        if (!compensated || !m.ring_lo) return cudaErrorInvalidValue;
        return launch_impl<true, false, true>(m, s, items, nitems, pp, err, part, comp_sq, sc, st, grid_warps);
    }
    if (compensated)
        return launch_impl<true, false, false>(m, s, items, nitems, pp, err, part, comp_sq, sc, st, grid_warps);
    return launch_impl<false, false, false>(m, s, items, nitems, pp, err, part, comp_sq, sc, st, grid_warps);
}

}  // namespace pbng
