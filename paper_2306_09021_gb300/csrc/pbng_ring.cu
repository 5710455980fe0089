// Ring-layout colour pass and residual for sm_103a.
//
// Layout: every free vertex of a colour owns W consecutive record slots
// (W = 4, 8, 16 or 32: the smallest power of two holding both its incident
// tets and its 1-ring, the distinct vertices it shares a tet with).  Slot l
// holds one incident tet (dN/dX of the other three vertices, 2 mu V,
// lambda V, and the three vertices' positions in the 1-ring as bytes) and the
// id of the l-th 1-ring vertex.  A warp's work item is 32 aligned slots =
// 32 / W vertices, one W-lane group each.
//
// Each warp is persistent and runs its own three-stage pipeline, with no
// block-wide barrier anywhere:
//   * lane 0 fetches an item's records and 1-ring ids (one RingBlock) with a
//     TMA 1D bulk copy (cp.async.bulk ... mbarrier::complete_tx) two items ahead;
//   * once they land, every lane gathers the displacement pair of its 1-ring
//     vertex (and the item's own vertices and aux data) with cp.async one item
//     ahead, so each neighbour is read once per vertex update, not once per
//     incident tet;
//   * the compute forms u_j - u_i once per 1-ring vertex, passes the three a
//     tet needs to its lane by warp shuffles, evaluates the element term
//     (pbng_element.cuh), sums the W lanes and adds the vertex terms; the
//     group's first lane queues the vertex's force and Hessian;
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

#include <stdint.h>

#include <type_traits>

namespace pbng {
namespace {

using el::f3;
using el::kFull;
using namespace async;

constexpr int kWarps = kBlock / 32;
// Three record stages (items requested two ahead) and 3 CTAs of 8 warps per
// SM: with two stages and 4 CTAs (64 registers) the passes were 15 % slower,
// the shorter pipeline exposing more TMA latency than the extra warps hide.
constexpr int kRecStages = 3;                 // record stages; items are requested kRecStages - 1 ahead
constexpr int kRecAhead = kRecStages - 1;
constexpr int kGatStages = 2;
constexpr int kItemVerts = kRingLanes / 4;
constexpr int kCtasPerSm = 3;
// Extended-precision passes (float-float element forces) need more registers
// than 3 CTAs of 8 warps leave.
constexpr int kCtasPerSmExt = 2;
constexpr int kQueue = 32;   // deferred vertex updates per warp

using RecStage = RingBlock;
static_assert(kRingLanes == 32, "one RingBlock per ring item");

struct __align__(16) GatStage {
    float4 nh[kRingLanes];   // 1-ring displacement hi
    float4 nl[kRingLanes];   // 1-ring displacement lo
    float4 oh[kItemVerts];   // own vertex hi
    float4 ol[kItemVerts];   // own vertex lo
    float4 a0[kItemVerts];   // aux0 (f_ext, K), residual passes only
    float4 a1[kItemVerts];   // aux1 (spring target, n.X - d), residual passes only
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

struct __align__(16) WarpSmem {
    RecStage rec[kRecStages];
    GatStage gat[kGatStages];
    UpdQueue q;
    Item desc[kRecStages];
    unsigned long long bar[kRecStages];
};

static_assert(kCtasPerSm * (kWarps * sizeof(WarpSmem) + 1024) <= 228 * 1024,
              "the per-warp stages of kCtasPerSm CTAs exceed an SM's shared memory");

// Extended-precision passes also stage the low words of the item's records
// (RingLoBlock), gathered with the 1-ring one item ahead.
struct __align__(16) LoStage {
    float4 la[kRingLanes];
    float4 lb[kRingLanes];
    float4 lc[kRingLanes];
};
struct __align__(16) WarpSmemExt : WarpSmem {
    LoStage lo[kGatStages];
};
static_assert(kCtasPerSmExt * (kWarps * sizeof(WarpSmemExt) + 1024) <= 228 * 1024,
              "the per-warp stages of kCtasPerSmExt extended CTAs exceed an SM's shared memory");

template <bool EXT>
using SmemOf = typename std::conditional<EXT, WarpSmemExt, WarpSmem>::type;

constexpr int kRecBytes = (int)sizeof(RingBlock);
static_assert(kRecBytes % 16 == 0, "bulk copies move multiples of 16 bytes");

// Lane 0: request the records and 1-ring ids of item `it` into stage r.  An
// item whose whole component is frozen is marked skipped and fetches nothing.
// `extra` bytes are expected beyond the copy (the timeout test hook).
__device__ __forceinline__ void issue_records(const DeviceMesh& m, Item it, WarpSmem& S, int r,
                                              uint32_t extra = 0u) {
    it.skip = (it.comp >= 0 && m.comp_active && !m.comp_active[it.comp]) ? 1 : 0;
    S.desc[r] = it;
    unsigned long long* bar = S.bar + r;
    if (it.skip) {
        mbar_arrive_expect_tx(bar, 0);
        return;
    }
    mbar_arrive_expect_tx(bar, kRecBytes + extra);
    bulk_g2s(&S.rec[r], m.ring + (it.slot0 >> 5), kRecBytes, bar);
}

// All lanes: gather the 1-ring displacements and own-vertex data of the item
// in record stage r into gather stage g.  AUX: also the vertices' aux data
// (passes that add the vertex terms when the element sums are done).
template <bool COMP, bool AUX, typename SM>
__device__ __forceinline__ void issue_gathers(const DeviceMesh& m, const State& s, SM& S, int r, int g,
                                              int lane) {
    const Item it = S.desc[r];
    if (it.skip) return;
    GatStage& G = S.gat[g];
    const int id = S.rec[r].id[lane];
    cp_async16(G.nh + lane, s.hi + id);
    if (COMP) cp_async16(G.nl + lane, s.lo + id);
    if (lane < it.nv) {
        const int v = it.v0 + lane;
        cp_async16(G.oh + lane, s.hi + v);
        if (COMP) cp_async16(G.ol + lane, s.lo + v);
        if (AUX) {  // the float32 update passes add the vertex terms when the queue is flushed
            cp_async16(G.a0 + lane, m.aux0 + v);
            cp_async16(G.a1 + lane, m.aux1 + v);
        }
    }
    if constexpr (std::is_same<SM, WarpSmemExt>::value) {
        const RingLoBlock& L = m.ring_lo[it.slot0 >> 5];
        cp_async16(S.lo[g].la + lane, L.la + lane);
        cp_async16(S.lo[g].lb + lane, L.lb + lane);
        cp_async16(S.lo[g].lc + lane, L.lc + lane);
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
template <int W, bool UPDATE, int MODEL>
__device__ __forceinline__ void compute_item_ext(const DeviceMesh& m, State s, WarpSmemExt& S, const Item& it, int r,
                                                 int g, int lane, PassParams pp, int32_t* err, double& rr,
                                                 double* comp_sq) {
    const RecStage& R = S.rec[r];
    const GatStage& G = S.gat[g];
    const int j = lane / W;
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
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = el::group_sum_ff<W>(f[k]);
    if (UPDATE) {
#pragma unroll
        for (int k = 0; k < 6; ++k) A[k] = el::group_sum<W>(A[k]);
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

template <int W, bool COMP, bool UPDATE, int MODEL>
__device__ __forceinline__ void compute_item_w(const DeviceMesh& m, State s, WarpSmem& S, const Item& it, int r,
                                               int g, int lane, uint32_t btab, int qn, double& rr,
                                               double* comp_sq) {
    const RecStage& R = S.rec[r];
    const GatStage& G = S.gat[g];
    const int j = lane / W;
    const bool active = j < it.nv;
    const float3 zero3 = make_float3(0.f, 0.f, 0.f);
    float3 uh = zero3, ul = zero3, d = zero3;
    if (active) {
        uh = f3(G.oh[j]);
        if (COMP) ul = f3(G.ol[j]);
        d = el::pair_diff<COMP>(G.nh[lane], COMP ? G.nl[lane] : make_float4(0.f, 0.f, 0.f, 0.f), uh, ul);
    }
    const float4 ra = R.ra[lane], rb = R.rb[lane], rc = R.rc[lane];
    const int loc = __float_as_int(rc.w);
    const int base = lane & ~(W - 1);
    const int s1 = base + (loc & 255), s2 = base + ((loc >> 8) & 255), s3 = base + ((loc >> 16) & 255);
    const float3 d1 = make_float3(__shfl_sync(kFull, d.x, s1), __shfl_sync(kFull, d.y, s1), __shfl_sync(kFull, d.z, s1));
    const float3 d2 = make_float3(__shfl_sync(kFull, d.x, s2), __shfl_sync(kFull, d.y, s2), __shfl_sync(kFull, d.z, s2));
    const float3 d3 = make_float3(__shfl_sync(kFull, d.x, s3), __shfl_sync(kFull, d.y, s3), __shfl_sync(kFull, d.z, s3));
    float rv[3] = {0.f, 0.f, 0.f};
    float A[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    el::element_math_m<UPDATE, MODEL, false>(f3(ra), f3(rb), f3(rc), ra.w, rb.w, d1, d2, d3, rv, A);
    if constexpr (UPDATE) {
        // the element sums of the group's vertex go straight into the queue
        // from the lanes that hold them; the vertex terms are added at flush
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
        // the element terms of the lane in float32, their W-lane sum and the
        // vertex terms in float-float
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

// The lane width is uniform over an item: dispatch once per item.
template <bool COMP, bool UPDATE, int MODEL, bool EXT>
__device__ __forceinline__ void compute_item(const DeviceMesh& m, State s, SmemOf<EXT>& S, const Item& it, int r,
                                             int g, int lane, uint32_t btab, int qn, double& rr, double* comp_sq,
                                             PassParams pp, int32_t* err) {
    if (it.skip) return;  // uniform over the warp
    if constexpr (EXT) {
        switch (it.w) {
            case 4: compute_item_ext<4, UPDATE, MODEL>(m, s, S, it, r, g, lane, pp, err, rr, comp_sq); break;
            case 8: compute_item_ext<8, UPDATE, MODEL>(m, s, S, it, r, g, lane, pp, err, rr, comp_sq); break;
            case 16: compute_item_ext<16, UPDATE, MODEL>(m, s, S, it, r, g, lane, pp, err, rr, comp_sq); break;
            default: compute_item_ext<32, UPDATE, MODEL>(m, s, S, it, r, g, lane, pp, err, rr, comp_sq); break;
        }
        return;
    }
    switch (it.w) {
        case 4: compute_item_w<4, COMP, UPDATE, MODEL>(m, s, S, it, r, g, lane, btab, qn, rr, comp_sq); break;
        case 8: compute_item_w<8, COMP, UPDATE, MODEL>(m, s, S, it, r, g, lane, btab, qn, rr, comp_sq); break;
        case 16: compute_item_w<16, COMP, UPDATE, MODEL>(m, s, S, it, r, g, lane, btab, qn, rr, comp_sq); break;
        default: compute_item_w<32, COMP, UPDATE, MODEL>(m, s, S, it, r, g, lane, btab, qn, rr, comp_sq); break;
    }
}

// All lanes: solve and write the qn queued vertices, one per lane.  The own
// displacement is read again here; no other update of the pass writes it.
template <bool COMP>
__device__ __forceinline__ void flush_queue(const DeviceMesh& m, State s, const WarpSmem& S, int qn, int lane,
                                            PassParams pp, int32_t* err) {
    __syncwarp();
    if (lane < qn) {
        const int v = S.q.v[lane];
        if (v >= 0) {
            float rv[3], A[6];
#pragma unroll
            for (int k = 0; k < 3; ++k) rv[k] = S.q.val[k][lane];
#pragma unroll
            for (int k = 0; k < 6; ++k) A[k] = S.q.val[3 + k][lane];
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
// EXT: extended precision (compute_item_ext; COMP must be true).
template <bool COMP, bool UPDATE, int MODEL, bool EXT>
__global__ void __launch_bounds__(kBlock, EXT ? kCtasPerSmExt : kCtasPerSm)
    ring_kernel(const DeviceMesh m, State s, const Item* __restrict__ items, int nitems, PassParams pp,
                int32_t* err, double* partial, double* comp_sq, int blocked) {
    static_assert(!EXT || COMP, "extended precision keeps the iterate as a float pair");
    constexpr bool AUX = !UPDATE || EXT;
    constexpr bool QUEUE = UPDATE && !EXT;
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_release();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SmemOf<EXT>& S = reinterpret_cast<SmemOf<EXT>*>(smem)[warp];
    const int gw = (int)blockIdx.x * kWarps + warp, nw = (int)gridDim.x * kWarps;
    int n, first, stride;
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
    double rr = 0.0;
    const uint32_t btab = QUEUE ? butterfly_table(lane) : 0u;
    int qn = 0;                  // queued vertex updates (warp-uniform)
    int issued = 0, waited = 0;  // items whose records were requested / awaited
    bool ok = true;
    Item next{};                 // lane 0: next item to request, loaded one item early
    if (n > 0) {
        if (lane == 0) {
            for (int i = 0; i < kRecStages; ++i) mbar_init(S.bar + i, 1);
            fence_mbar_init();
            for (int i = 0; i < kRecAhead && i < n; ++i)
                issue_records(m, items[first + i * stride], S, i, i == 0 ? (uint32_t)m.copy_shortfall : 0u);
            if (n > kRecAhead) next = items[first + kRecAhead * stride];
        }
        issued = n < kRecAhead ? n : kRecAhead;
        __syncwarp();
        // Records, items and component flags are written by no kernel; the
        // iterate read from here on is written by the previous kernel.
        pdl_wait();
        ok = mbar_wait(S.bar + 0, 0);
        waited = ok ? 1 : 0;  // a stage whose wait gave up is drained again on abort
        if (__any_sync(kFull, !ok)) goto abort;
        issue_gathers<COMP, AUX>(m, s, S, 0, 0, lane);
        cp_async_commit();
        for (int k = 0; k < n; ++k) {
            // Record stage (k + kRecAhead) % kRecStages and gather stage
            // (k+1)%2 were last read by item k-1, finished before the previous
            // __syncwarp.
            if (k + kRecAhead < n) {
                if (lane == 0) {
                    fence_proxy_async();
                    issue_records(m, next, S, (k + kRecAhead) % kRecStages);
                    if (k + kRecAhead + 1 < n) next = items[first + (k + kRecAhead + 1) * stride];
                }
                issued = k + kRecAhead + 1;
            }
            ok = true;
            if (k + 1 < n) {
                ok = mbar_wait(S.bar + (k + 1) % kRecStages, ((k + 1) / kRecStages) & 1);
                waited = ok ? k + 2 : k + 1;
                if (ok) issue_gathers<COMP, AUX>(m, s, S, (k + 1) % kRecStages, (k + 1) % kGatStages, lane);
            }
            cp_async_commit();
            cp_async_wait<1>();  // this lane's gathers of item k have landed
            if (__any_sync(kFull, !ok)) goto abort;
            __syncwarp();        // ... and the other lanes'
            const Item it = S.desc[k % kRecStages];
            compute_item<COMP, UPDATE, MODEL, EXT>(m, s, S, it, k % kRecStages, k % kGatStages, lane, btab, qn, rr,
                                                   comp_sq, pp, err);
            if (QUEUE) {
                if (!it.skip) qn += it.nv;
                if (qn > kQueue - kItemVerts || (k + 1 == n && qn > 0)) {
                    flush_queue<COMP>(m, s, S, qn, lane, pp, err);
                    qn = 0;
                }
            }
            __syncwarp();
        }
    }
    if (!UPDATE && partial) {
        if (n == 0) pdl_wait();  // idle warp: order its write after the predecessor
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) rr += __shfl_xor_sync(kFull, rr, off);
        if (lane == 0) partial[gw] = rr;
    }
    return;

abort:
    // A record copy did not complete in time: report it, let the copies this
    // warp started finish (bounded), then leave.
    if (lane == 0) {
        atomicOr(err, kErrTimeout);
        for (int k = waited; k < issued; ++k) (void)mbar_wait(S.bar + k % kRecStages, (k / kRecStages) & 1);
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

int ring_ctas(int nitems, int ctas_per_sm, int balanced = 0, int max_cps = kCtasPerSm) {
    const int want = (nitems + kWarps - 1) / kWarps;
    const int cps = ctas_per_sm < 1 ? 1 : (ctas_per_sm > max_cps ? max_cps : ctas_per_sm);
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

template <bool COMP, bool UPDATE, bool EXT = false>
cudaError_t launch_impl(const DeviceMesh& m, State s, const Item* items, int nitems, PassParams pp,
                        int32_t* err, double* partial, double* comp_sq, RingSched sc, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const int bytes = kWarps * (int)sizeof(SmemOf<EXT>);  // attribute set by ring_prepare()
    // An extended residual writes the partials of the float32 residual's grid
    // (2 CTAs per SM are resident, the rest follow); an extended update pass
    // keeps its grid to what is resident.
    const int grid = ring_ctas(nitems, sc.ctas_per_sm, sc.balanced, (EXT && UPDATE) ? kCtasPerSmExt : kCtasPerSm);
    if (pp.model == el::kNeoHookean)
        return launch_kernel(ring_kernel<COMP, UPDATE, el::kNeoHookean, EXT>, grid, kBlock, bytes, st, m, s, items,
                             nitems, pp, err, partial, comp_sq, sc.blocked);
    if (pp.model == el::kStableNeoHookean)
        return launch_kernel(ring_kernel<COMP, UPDATE, el::kStableNeoHookean, EXT>, grid, kBlock, bytes, st, m, s,
                             items, nitems, pp, err, partial, comp_sq, sc.blocked);
    return launch_kernel(ring_kernel<COMP, UPDATE, el::kCorotated, EXT>, grid, kBlock, bytes, st, m, s, items, nitems,
                         pp, err, partial, comp_sq, sc.blocked);
}

}  // namespace

int ring_warps(int nitems) { return nitems > 0 ? ring_ctas(nitems, kCtasPerSm) * kWarps : 0; }

int ring_max_ctas_per_sm() { return kCtasPerSm; }

cudaError_t ring_prepare() {
    // Three CTAs of 8 warps with their per-warp stages and queues need almost
    // all of an SM's shared memory: ask for the largest carveout.
    const int bytes = kWarps * (int)sizeof(WarpSmem), bytes_ext = kWarps * (int)sizeof(WarpSmemExt);
    const void* fns[18] = {
        (const void*)ring_kernel<true, true, 0, false>,  (const void*)ring_kernel<false, true, 0, false>,
        (const void*)ring_kernel<true, false, 0, false>, (const void*)ring_kernel<false, false, 0, false>,
        (const void*)ring_kernel<true, true, 1, false>,  (const void*)ring_kernel<false, true, 1, false>,
        (const void*)ring_kernel<true, false, 1, false>, (const void*)ring_kernel<false, false, 1, false>,
        (const void*)ring_kernel<true, true, 2, false>,  (const void*)ring_kernel<false, true, 2, false>,
        (const void*)ring_kernel<true, false, 2, false>, (const void*)ring_kernel<false, false, 2, false>,
        (const void*)ring_kernel<true, true, 0, true>,   (const void*)ring_kernel<true, false, 0, true>,
        (const void*)ring_kernel<true, true, 1, true>,   (const void*)ring_kernel<true, false, 1, true>,
        (const void*)ring_kernel<true, true, 2, true>,   (const void*)ring_kernel<true, false, 2, true>};
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
    if (compensated) return launch_impl<true, true>(m, s, items, nitems, p, err, nullptr, nullptr, sc, st);
    return launch_impl<false, true>(m, s, items, nitems, p, err, nullptr, nullptr, sc, st);
}

cudaError_t launch_ring_residual(const DeviceMesh& m, State s, const Item* items, int nitems,
                                 bool compensated, double* warp_partial, double* comp_sq, int model, int32_t* err,
                                 cudaStream_t st, bool extended) {
    const PassParams pp{1.f, 0.f, model};
    const RingSched sc{kCtasPerSm, 0, 0};  // ring_warps() partials
    double* part = comp_sq ? nullptr : warp_partial;
    if (extended) {
        if (!compensated || !m.ring_lo) return cudaErrorInvalidValue;
        return launch_impl<true, false, true>(m, s, items, nitems, pp, err, part, comp_sq, sc, st);
    }
    if (compensated) return launch_impl<true, false>(m, s, items, nitems, pp, err, part, comp_sq, sc, st);
    return launch_impl<false, false>(m, s, items, nitems, pp, err, part, comp_sq, sc, st);
}

}  // namespace pbng
