// Internal declarations shared by the host runtime (pbng_api.cpp) and the
// CUDA kernels (pbng_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pbng {

// A run of free vertices (internal, colour-ordered ids) that share a lane
// group width: each vertex gets `width` consecutive lanes of one warp.
struct Segment {
    int32_t v_begin;
    int32_t v_end;
    int32_t width;        // 4, 8, 16 or 32
    int32_t block_begin;  // first block of this segment within its launch
};

constexpr int kMaxSegments = 48;
constexpr int kBlock = 256;

struct SegmentTable {
    int32_t count;
    int32_t total_blocks;
    Segment seg[kMaxSegments];
};

// Device view of a prepared mesh.  Per-incidence records are laid out in the
// order the colour passes consume them (vertex-major CSR over the internal,
// colour-ordered free vertices), so consecutive lanes read consecutive
// records.
// The records of one 32-slot ring item, contiguous so that one bulk copy
// fetches them.
struct __align__(16) RingBlock {
    float4 ra[32];   // g_j1 (xyz), a = 2 mu V
    float4 rb[32];   // g_j2 (xyz), b = lambda V
    float4 rc[32];   // g_j3 (xyz), local ring indices l1 | l2 << 8 | l3 << 16 (int bits)
    int32_t id[32];  // internal id of the vertex's l-th 1-ring neighbour (own id when padding)
};

// Low words of the same slots (extended precision, PBNG_PREC_EXTENDED):
// each record value x is held as the float pair hi + lo with hi the RingBlock
// entry and lo = x - hi, so that the element constants keep about 48 bits.
struct __align__(16) RingLoBlock {
    float4 la[32];   // g_j1 low words (xyz), a low word
    float4 lb[32];   // g_j2 low words (xyz), b low word
    float4 lc[32];   // g_j3 low words (xyz), 0
};

// Float32 passes (pbng_ring.cu): one 32-lane pair item.  A vertex of pair
// width W owns W consecutive lanes, W the smallest power of two (>= 4)
// holding half its incident tets and half its 1-ring.  Lane l of its group
// holds its 1-ring vertices l and W + l (PairIds) and two of its incident
// tets, A = tet l and B = tet W + l (PairRec; zero records where it has
// fewer).  The twelve values of a tet (g_j1, g_j2, g_j3, a = 2 mu V,
// b = lambda V, and the slots of its three other vertices among the item's
// 64 1-ring slots as bytes, int bits) are interleaved so that value k of tet
// A and of tet B are adjacent words: (r[k/2][lane].x, .y) for even k and
// (.z, .w) for odd k, one operand of a packed f32x2 instruction.  1-ring
// vertex l of a group whose first lane is f sits in slot
// (l / W) 32 + f + (l % W).  Ids and records of an item are fetched by
// separate bulk copies: the ids one item earlier than the records.
struct __align__(16) PairRec {
    float4 r[6][32];
};
struct __align__(16) PairIds {
    int32_t id[2][32];  // 1-ring vertex ids of each lane (own id when padding)
};

struct DeviceMesh {
    int32_t nv;              // all vertices (free first, then clamped)
    int32_t nfree;
    const int32_t* inc_off;  // [nfree + 1] CSR offsets into the records
    const float4* rec_a;     // [ninc] other vertex ids j1, j2, j3 (int bits), a = 2 mu V
    const float4* rec_b;     // [ninc] g_j1 (xyz), b = lambda V
    const float4* rec_c;     // [ninc] g_j2 (xyz), g_j3.x
    const float2* rec_d;     // [ninc] g_j3.y, g_j3.z
    const float4* aux0;      // [nfree] f_ext (xyz), total spring stiffness K
    const float4* aux1;      // [nfree] spring target displacement (xyz), n.X - d
    const float4* aux_lo;    // [nfree] low words of f_ext (xyz): f_ext = aux0 + aux_lo
    const int32_t* comp;     // [nfree] component id, or nullptr for one component
    const int32_t* comp_active;  // [ncomp] 0 = frozen (converged), or nullptr
    // Residuals of several components: each free vertex's |r|^2 goes to
    // vsq[v] and the per-component sums follow in a fixed order
    // (launch_comp_reduce); nullptr: atomic per-component sums instead.
    double* vsq;
    // Extended residual only (nullptr otherwise): each free vertex's
    // float-float force f + f^ext as fout_hi[v] + fout_lo[v] (xyz).
    float4* fout_hi;
    float4* fout_lo;
    // Ring layout (colours whose vertices all fit 32 lanes): one 32-slot
    // item per warp; vertex v of a lane-width-W run owns W consecutive slots.
    // Slot s is entry s % 32 of block s / 32 (RingBlock).
    const struct RingBlock* ring;  // [nslots / 32]
    const struct RingLoBlock* ring_lo;  // [nslots / 32] low words of the same records
    // The same colours in pair items (float32 passes and residuals): one
    // PairRec and one PairIds per item of the pair item list.
    const struct PairRec* prec;
    const struct PairIds* pids;
    // Test hook (pbng_test_set_copy_shortfall): bytes that each warp's first
    // bulk copy of a ring pass (records, or a pair item's ids) is expected to
    // carry beyond its size, so that its bounded wait runs out; 0 in normal use.
    int32_t copy_shortfall;
    float pn_x, pn_y, pn_z;  // contact plane normal (unit)
    float k_contact;         // 0 = no plane
    // General weak constraints (nullptr when there are none): constraint c
    // couples up to 8 vertices wc_v[8c + q] (internal ids, -1 unused) with
    // coefficients wc_b[8c + q] = w0 - w1; C = C0 + sum_q b_q u_q with the
    // rest value C0 = sum_q b_q X_q as a float pair wc_c0[2c] + wc_c0[2c + 1];
    // stiffness upper triangle wc_k[6c ..].  Free vertex v owns entries
    // wc_off[v] .. wc_off[v + 1] of wc_list = (constraint, own coefficient bits).
    const int32_t* wc_off;
    const int2* wc_list;
    const int32_t* wc_v;
    const float* wc_b;
    const float* wc_k;
    const float4* wc_c0;
};

// The iterate: displacement u = x - X as a float pair hi + lo (lo is unused
// in plain FP32 mode).  xyz used, w = 0.
struct State {
    float4* hi;
    float4* lo;
};

struct PassParams {
    float step;       // scale of the Newton step
    float skip_tol;   // 0 = never skip
    int model;        // constitutive model: 0 corotated, 1 Neo-Hookean, 2 stable Neo-Hookean
};

// Error bits written by the kernels (OR-ed into a device word).
enum : int32_t {
    kErrNonSPD = 1,      // det(A_i) <= 0 or non-finite
    kErrNonFinite = 2,   // non-finite update
    kErrTimeout = 4,     // a bounded wait on an asynchronous copy gave up
};

// One warp's work item in the ring layout: 32 slots starting at slot0,
// holding nv = 32 / w (or fewer at the end of a run) vertices v0, v0+1, ...
struct Item {
    int32_t v0;
    int32_t nv;
    int32_t w;
    int32_t slot0;
    int32_t comp;  // component of every vertex of the item, or -1 when mixed
    int32_t skip;  // set on the device copy: the item's component is frozen
    int32_t pad[2];
};
constexpr int kRingLanes = 32;

// Host launch wrappers (pbng_kernels.cu).  All enqueue on `st`.
// Programmatic dependent launch for the sweep kernels (colour passes,
// acceleration, residual): on while a chunk of sweeps is captured into a
// graph, off for plain launches (timed per launch with events) and for
// everything else.  Per host thread; PdlScope restores the previous value.
void set_pdl(bool on);
bool pdl_enabled();
struct PdlScope {
    bool old;
    explicit PdlScope(bool on) : old(pdl_enabled()) { set_pdl(on); }
    ~PdlScope() { set_pdl(old); }
    PdlScope(const PdlScope&) = delete;
    PdlScope& operator=(const PdlScope&) = delete;
};

cudaError_t launch_colour_pass(const DeviceMesh& m, State s, const SegmentTable& t, PassParams p,
                               bool compensated, int32_t* err, cudaStream_t st);
cudaError_t launch_residual(const DeviceMesh& m, State s, const SegmentTable& t, bool compensated,
                            double* block_partial, double* comp_sq, int32_t ncomp,
                            float* r_out, int model, cudaStream_t st);
cudaError_t launch_reduce(const double* partial, int32_t n, double* out, cudaStream_t st);
// out[c] = sum of vsq[list[k]] for k in off[c] .. off[c + 1], in a fixed order.
cudaError_t launch_comp_reduce(int32_t ncomp, const int32_t* off, const int32_t* list, const double* vsq,
                               double* out, cudaStream_t st);
cudaError_t launch_accel(int32_t nfree, State cur, State p1, State p2, const float2* wg,
                         const int32_t* comp, const int32_t* comp_active, bool compensated, cudaStream_t st);
cudaError_t launch_load(int32_t nv, int32_t nfree, const float* u_user, const int32_t* perm,
                        const float4* dir_hi, const float4* dir_lo, State s, cudaStream_t st);
cudaError_t launch_store(int32_t nv, const int32_t* perm, State s, float* u_user, cudaStream_t st);
cudaError_t launch_copy_state(int32_t n, State src, State dst, cudaStream_t st);
// Backward-Euler step setup (Eq. fem_be): for free vertex v (internal order)
// with caller id o = perm[v], uhat = 2 u[o] - u_prev[o]; the inertia acts as
// a zero-rest spring of stiffness k_v = m_v / dt^2 to uhat, merged with the
// vertex's own springs into aux; u[o] becomes the predictor
// uhat + f_ext / k_v and u_prev[o] the old u[o] (every vertex).
cudaError_t launch_inertia(int32_t nv, int32_t nfree, const int32_t* perm, float* u, float* u_prev,
                           const float4* base0, const float4* base1, const float* k, float4* aux0, float4* aux1,
                           cudaStream_t st);

// Ring-layout kernels (pbng_ring.cu): persistent warps, each streaming its
// items with TMA bulk copies and cp.async gathers.  Float32 passes and
// residuals (extended = false) take the pair item list (PairRec, PairIds),
// extended ones the ring item list (RingBlock records and their low words).
// A residual runs a grid of exactly grid_warps warps (a multiple of 8, at
// least ring_warps() of its item list) and writes one FP64 partial per warp,
// or, with comp_sq, per-component sums.
// A colour pass's launch schedule: CTAs per SM of the persistent grid
// (1..ring_max_ctas_per_sm()), the item order (0 strided, 1 blocked), and
// whether the grid is trimmed to the fewest warps that take the same number
// of item rounds (1 balanced), so that no warp idles through the last round.
struct RingSched {
    int ctas_per_sm;
    int blocked;
    int balanced;
};
int ring_warps(int nitems);
int ring_max_ctas_per_sm();
cudaError_t ring_prepare();  // sets kernel attributes (call outside stream capture)
// extended: float-float element forces from the float-pair records (needs
// compensated and ring_lo), summed in float-float (pbng_ff.cuh).
cudaError_t launch_ring_pass(const DeviceMesh& m, State s, const Item* items, int nitems, PassParams p,
                             bool compensated, RingSched sc, int32_t* err, cudaStream_t st, bool extended = false);
cudaError_t launch_ring_residual(const DeviceMesh& m, State s, const Item* items, int nitems,
                                 bool compensated, double* warp_partial, double* comp_sq, int model,
                                 int32_t* err, cudaStream_t st, bool extended, int grid_warps);

// Equilibrium adjoint (pbng_adjoint.cu).  Vertex kernels: one warp per
// ring item; mode 0 computes the 3x3 diagonal blocks of H, mode 1 is one
// Gauss-Seidel pass over the given items (one colour), mode 2 writes one FP64
// partial of |dL/du - H lambda|^2 per warp (adjoint_warps(nitems) of them).
// Mode 3 writes r = f + f^ext at u to out and the SPD blocks of Eq. mod_hess
// to diag; mode 4 writes out = H lam (lam zero at clamped vertices); both
// write one FP64 partial per warp (|r|^2, lam . H lam).
enum { kAdjDiag = 0, kAdjSweep = 1, kAdjResid = 2, kAdjForce = 3, kAdjApply = 4 };
int adjoint_warps(int nitems);
cudaError_t launch_adjoint_vertex(int mode, const DeviceMesh& m, State u, float4* lam, const float4* gv,
                                  float4* diag, const Item* items, int nitems, int32_t* err, double* partial,
                                  cudaStream_t st, float4* out = nullptr, int model = 0);
// The block Gauss-Seidel pass (mode 1) of one ring colour, pipelined like the
// colour pass; adjoint_prepare sets its kernel attributes (call outside
// stream capture).
cudaError_t launch_adjoint_ring_sweep(const DeviceMesh& m, State u, float4* lam, const float4* gv, const float4* diag,
                                      const Item* items, int nitems, int32_t* err, int model, cudaStream_t st);
cudaError_t adjoint_prepare();
// The Hessian action out = H lam with the same pipeline, over any items (all
// colours in one launch; lam is only read), one FP64 partial of
// lam . H lam per warp of its grid (adjoint_ring_apply_warps(nitems)).
int adjoint_ring_apply_warps(int nitems);
cudaError_t launch_adjoint_ring_apply(const DeviceMesh& m, State u, const float4* lam, const Item* items, int nitems,
                                      int32_t* err, int model, float4* out, double* partial, cudaStream_t st);

// Preconditioned conjugate gradients on the free rows (pbng_adjoint.cu): the
// scalars stay on the device in sc[0..3] = (r.z, p.Hp, new r.z, |r|^2); one
// FP64 partial per kBlock threads (vec_blocks(n) of them).
int vec_blocks(int n);
cudaError_t launch_cg_init(int n, const float4* r, const float4* diag, float4* x, float4* z, float4* p,
                           double* partial, cudaStream_t st);
cudaError_t launch_cg_update(int n, const double* sc, float4* x, float4* r, const float4* p, const float4* q,
                             const float4* diag, float4* z, double* part_rz, double* part_rr, int32_t* flag,
                             cudaStream_t st);
cudaError_t launch_cg_dir(int n, const double* sc, const float4* z, float4* p, const int32_t* flag, double* sc_rw,
                          cudaStream_t st);
cudaError_t launch_newton_axpy(int nv, int nfree, State src, const float4* x, float s, State dst, cudaStream_t st);
cudaError_t launch_gather_vec(int nv, int nfree, const int32_t* perm, const float* in, float4* out, cudaStream_t st);
cudaError_t launch_scatter_vec(int nv, int nfree, const int32_t* perm, const float4* in, float* out, cudaStream_t st);
cudaError_t launch_adjoint_tets(int ne, int nfree, const int4* tv, const float4* tb, State u, const float4* lam,
                                float* dLdlogE, float* hdl, cudaStream_t st, int model = 0);
cudaError_t launch_gather_rhs(int nfree, const int32_t* perm, const float* dLdu, float4* gv, cudaStream_t st);
// Refined adjoint (pbng_adjoint in extended precision), pbng_adjoint.cu:
// u_plus / u_minus = u +- eps (lam_hi + lam_lo) over all nv vertices (lam is
// zero at clamped ones), in float-float;
cudaError_t launch_adjoint_shift(int nv, State u, const float4* lam_hi, const float4* lam_lo, float eps, State up,
                                 State um, cudaStream_t st);
// rhs[w] = gv[w] + (F+ - F-)[w] / (2 eps) (that is dL/du - H lam, H = -dF/du
// by central differences of the float-float force), FP64 |rhs|^2 per block
// into partial (adj_vec_blocks(nfree) of them);
int adj_vec_blocks(int n);
cudaError_t launch_adjoint_refine_rhs(int nfree, const float4* gv, const float4* fp_hi, const float4* fp_lo,
                                      const float4* fm_hi, const float4* fm_lo, double inv2eps, float4* rhs,
                                      double* partial, cudaStream_t st);
// lam_hi + lam_lo += d (float-float), and the largest |component| of the sum
// into *maxabs (float bits; zero it first).
cudaError_t launch_adjoint_accumulate(int nfree, const float4* d, float4* lam_hi, float4* lam_lo, float* maxabs,
                                      cudaStream_t st);
// Conjugate gradients on the adjoint system (PBNG_ACCEL_CG), n free rows,
// one FP64 partial per block (adj_vec_blocks(n) of them), the scalars on the
// device as in launch_cg_update (sc[0] = r . z, sc[1] = p . H p,
// sc[2] = the new r . z): x += a p and r -= a q with a = sc[0] / sc[1] and
// |r|^2 partials (a non-positive p . H p sets *flag and changes nothing);
// r . z partials.  The direction update is launch_cg_dir.
cudaError_t launch_acg_step(int n, const double* sc, int32_t* flag, const float4* p, const float4* q, float4* x,
                            float4* r, double* partial, cudaStream_t st);
cudaError_t launch_acg_dot(int n, const float4* r, const float4* z, double* partial, cudaStream_t st);
// The two-sided weak constraints' part of H_DF lam (into hdl, float4 rows).
cudaError_t launch_adjoint_weak_clamped(int nwc, int nfree, const DeviceMesh& m, const float4* lam, float* hdl,
                                        cudaStream_t st);
cudaError_t launch_clamped_grad(int nd, const int32_t* dq_internal, const int32_t* dq_caller, const float* dLdu,
                                const float* hdl, float* out, cudaStream_t st);

// FP32 FMA throughput probe (pbng_kernels.cu): one launch of `blocks` CTAs
// of 256 threads, each running `iters` rounds of independent FMA chains into
// out[blocks * 256], bracketed by events e0 / e1 on st; *flops = the flops
// it executes.
cudaError_t fma_peak(cudaStream_t st, float* out, int blocks, int iters, cudaEvent_t e0, cudaEvent_t e1,
                     double* flops);

// Fixed device scratch of the allocation-free residual (pbng_kernels.cu).
int noalloc_scratch_capacity();
cudaError_t noalloc_scratch(int device, double** out);

}  // namespace pbng
