// Host runtime and C ABI of the PBNG library (declared in include/pbng.h).
//
// Mesh preparation (per-tet dN/dX, rest volume and Lame parameters), the
// greedy node colouring, the colour-ordered device layout and the sweep
// driver live here; every per-sweep step runs in the kernels of
// pbng_kernels.cu.
#include "pbng.h"
#include "pbng_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <array>
#include <chrono>
#include <vector>

using namespace pbng;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct pbng_mesh {
    int device = 0;
    int32_t copy_shortfall = 0;  // pbng_test_set_copy_shortfall
    cudaStream_t stream = nullptr;
    int32_t nv = 0, ne = 0, ncomp = 1;
    std::vector<double> X;          // 3 nv
    std::vector<int32_t> tets;      // 4 ne
    std::vector<double> B;          // 9 ne, rows g_1..g_3 of Dm^{-1}
    std::vector<double> vol, mu, lam;
    std::vector<int32_t> comp_of;   // nv (empty = single component)

    // boundary data
    std::vector<uint8_t> is_dir;    // nv
    std::vector<double> dir_pos;    // 3 nv (valid where is_dir)
    std::vector<double> spr_K;      // nv, total spring stiffness
    std::vector<double> spr_KT;     // 3 nv, sum_s k_s t_s
    bool has_plane = false;
    double pn[3] = {0, 0, 1}, pd = 0.0, kc = 0.0;
    std::vector<double> fext;       // 3 nv
    // general weak constraints (pbng_set_weak_constraints), caller ids
    std::vector<std::vector<int32_t>> wc_v;
    std::vector<std::vector<double>> wc_b;
    std::vector<std::array<double, 6>> wc_k;
    bool wc_incremental = false;       // next layout: keep colours, revisit constraint vertices
    double colour_ms = 0.0, layout_ms = 0.0;

    // layout
    bool dirty = true;
    int32_t nfree = 0, ncol = 0;
    std::vector<int32_t> colour;    // nv, -1 clamped
    std::vector<int32_t> perm;      // internal -> caller id
    std::vector<SegmentTable> tables;  // one per colour
    std::vector<uint8_t> ring_colour;  // per colour: ring layout (else CSR, direct loads)
    bool all_ring = true;
    std::vector<Item> items;           // ring items, colour by colour
    std::vector<int32_t> item_off;     // ncol + 1 offsets into items
    int32_t nitems_ring = 0;
    std::vector<Item> pitems;          // pair items (float32 passes and residuals), colour by colour
    std::vector<int32_t> pitem_off;    // ncol + 1 offsets into pitems
    int32_t nitems_pair = 0;
    int32_t ring_partials = 0;         // residual partials of the ring launch (either item list)
    bool want_direct = false;          // params.kernel_path == 1 requested
    int model = 0;                     // constitutive model of the last sweep / solve (residuals use it)
    // backward Euler (pbng_set_inertia): dt > 0 and lumped masses, caller order
    double be_dt = 0.0;
    std::vector<double> be_mass;
    DevBuf d_aux_base0, d_aux_base1, d_be_k;  // aux without inertia, m_v / dt^2 (internal order)
    DevBuf d_wc_off, d_wc_list, d_wc_v, d_wc_b, d_wc_k, d_wc_c0;
    bool built_direct = false;         // layout built with want_direct
    std::vector<int32_t> table_partial_off;  // residual partial offset per colour
    int32_t total_partials = 0;
    pbng_solve_info info{};            // of the last pbng_solve
    std::vector<RingSched> sched;      // per colour launch schedule of the ring passes
    double tune_default_ms = 0.0, tune_ms = 0.0;
    int32_t tune_cands = 0;

    // device buffers
    DevBuf d_inc_off, d_rec_a, d_rec_b, d_rec_c, d_rec_d, d_aux0, d_aux1, d_aux_lo, d_comp, d_perm;
    DevBuf d_ring, d_ring_lo, d_items, d_prec, d_pids, d_pitems;
    DevBuf d_host_u;  // device copy of the caller's host iterate (pbng_sweep_host)
    DevBuf d_active;                   // int32 [ncomp] component flags (1 = active)
    DevBuf d_vsq, d_comp_off, d_comp_list;  // several components: per-vertex |r|^2, component -> vertices
    // adjoint (built on first use after each layout)
    DevBuf d_lam[3], d_gv, d_diag, d_hdl, d_tv, d_tb, d_dq_int, d_dq_caller, d_adj_partial;
    // refined adjoint (extended precision): multipliers as float pairs, the
    // correction's right-hand side, the forces at u +- eps lam, the shifted states
    DevBuf d_lam_hi, d_lam_lo, d_rhs, d_fp[4], d_shift[2][2], d_maxabs, d_refine_partial;
    // conjugate-gradient adjoint (PBNG_ACCEL_CG): residual r and H p, FP64 block partials
    DevBuf d_acg[2], d_acg_part[2], d_acg_sc;  // + device scalars (4 doubles and a flag)
    double h_min = 0.0;                // smallest rest element size (cube root of 6 V)
    // Newton-CG (pbng_newton_cg, pbng_force, pbng_hessian_apply): r, x, z, p, q
    DevBuf d_nw[5], d_nw_part[2], d_nw_sc, d_nw_flag;
    double* h_nw = nullptr;            // pinned: sc[3], flag
    bool adj_ready = false;
    std::vector<int32_t> dir_list;     // clamped ids in pbng_set_constraints order
    int32_t* h_active = nullptr;       // pinned host copy
    DevBuf d_dir_hi, d_dir_lo;
    DevBuf d_state[4][2];           // cur, p1, p2, tmp; hi/lo
    DevBuf d_partial, d_comp_sq, d_scalar, d_err;
    double* h_pinned = nullptr;     // ncomp + 2 doubles for readbacks; [ncomp] also carries the error flag
    DeviceMesh dm{};

    // iteration state
    bool has_state = false;
    int32_t sweep_l = 0;
    double omega_l = 1.0;
    int p1_slot = 1, p2_slot = 2;
    std::vector<double> r0;

    // captured chunks of sweeps (CUDA graphs), keyed by their configuration
    struct GraphEntry {
        int32_t K, accel, prec, with_res, p1, prof, model, order;
        float step, skip;
        cudaGraphExec_t exec = nullptr;
        int64_t nkernels = 0;
        std::vector<cudaEvent_t> ev;   // pairs around timed launches (profiled variant)
        std::vector<int> ev_kind;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap_stream = nullptr; // private stream the graphs are captured on
    DevBuf d_wg;                       // float2 [kMaxChunk] per-sweep acceleration weights
    float2* h_wg = nullptr;            // pinned staging for the weights of one call
    size_t h_wg_cap = 0;

    // profiling (pbng_set_profiling): event pairs per timed launch
    bool prof = false;
    struct EvPair { cudaEvent_t a, b; int kind; };
    std::vector<EvPair> ev_used;
    std::vector<cudaEvent_t> ev_free;
    int64_t prof_launches[3] = {0, 0, 0};   // colour pass, accel, residual
    double prof_ms[3] = {0, 0, 0};
    int64_t kernel_launches = 0;
    int64_t ninc = 0;

    std::string err;
};

namespace {

enum { kProfColour = 0, kProfAccel = 1, kProfResidual = 2 };

cudaError_t take_event(pbng_mesh* m, cudaEvent_t* e) {
    if (!m->ev_free.empty()) {
        *e = m->ev_free.back();
        m->ev_free.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

// Folds finished event pairs into the counters (synchronises the stream).
cudaError_t prof_flush(pbng_mesh* m) {
    if (m->ev_used.empty()) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return e;
    for (auto& p : m->ev_used) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) return e;
        m->prof_ms[p.kind] += ms;
        m->ev_free.push_back(p.a);
        m->ev_free.push_back(p.b);
    }
    m->ev_used.clear();
    return cudaSuccess;
}

// Records the opening event of a timed launch; returns its slot or -1.
int prof_begin(pbng_mesh* m, int kind) {
    if (!m->prof) return -1;
    if (m->ev_used.size() >= 8192 && prof_flush(m) != cudaSuccess) return -1;
    pbng_mesh::EvPair p{};
    p.kind = kind;
    if (take_event(m, &p.a) != cudaSuccess || take_event(m, &p.b) != cudaSuccess) return -1;
    if (cudaEventRecord(p.a, m->stream) != cudaSuccess) return -1;
    m->ev_used.push_back(p);
    return (int)m->ev_used.size() - 1;
}

void prof_end(pbng_mesh* m, int slot) {
    if (slot < 0) return;
    pbng_mesh::EvPair& p = m->ev_used[slot];
    cudaEventRecord(p.b, m->stream);
    m->prof_launches[p.kind]++;
}

pbng_status fail(pbng_mesh* m, pbng_status s, const std::string& msg) {
    if (m) m->err = msg;
    return s;
}

constexpr size_t kErrTextReserve = 512;

// For literal messages: assigning into the handle's reserved text buffer
// takes no host allocation (pbng_residual_noalloc relies on it).
pbng_status fail(pbng_mesh* m, pbng_status s, const char* msg) {
    if (m) m->err.assign(msg);
    return s;
}

pbng_status cuda_fail(pbng_mesh* m, cudaError_t e, const char* what) {
    return fail(m, PBNG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define PBNG_CUDA(m, call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(m, e_, #call); \
    } while (0)

void free_buf(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

constexpr int32_t kMaxChunk = 1024;
// Largest automatic Chebyshev rho (symmetric colour order).
constexpr double kRhoCap = 1.0 - 1e-6;

void destroy_graphs(pbng_mesh* m) {
    for (auto& g : m->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        for (cudaEvent_t e : g.ev) cudaEventDestroy(e);
    }
    m->graphs.clear();
}

cudaError_t ensure_buf(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return cudaSuccess;
    free_buf(b);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) b.bytes = bytes;
    return e;
}

template <class T>
cudaError_t upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
    cudaError_t e = ensure_buf(b, v.size() * sizeof(T));
    if (e != cudaSuccess || v.empty()) return e;
    e = cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);  // host vectors may go away after return
}

double det3(const double* F) {
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

// Section "Coloring and Parallelism" (node colouring): free vertices in
// ascending id take the least colour that no element containing them has
// registered yet, then register it in each of those elements.  Element
// colour sets are bit masks of `words` 64-bit words.
bool greedy_colour(const pbng_mesh& m, const std::vector<int32_t>& inc_off,
                   const std::vector<int32_t>& inc_tet, int32_t nelem, int words, std::vector<int32_t>& colour,
                   int32_t& ncol) {
    std::vector<uint64_t> used((size_t)nelem * words, 0);
    std::vector<uint64_t> acc(words);
    colour.assign(m.nv, -1);
    ncol = 0;
    for (int32_t i = 0; i < m.nv; ++i) {
        if (m.is_dir[i]) continue;
        std::fill(acc.begin(), acc.end(), 0);
        for (int32_t k = inc_off[i]; k < inc_off[i + 1]; ++k) {
            const uint64_t* u = &used[(size_t)inc_tet[k] * words];
            for (int w = 0; w < words; ++w) acc[w] |= u[w];
        }
        int c = -1;
        for (int w = 0; w < words && c < 0; ++w)
            if (~acc[w]) {
                uint64_t free_bits = ~acc[w];
                int b = 0;
                while (!(free_bits & 1ull)) { free_bits >>= 1; ++b; }
                c = 64 * w + b;
            }
        if (c < 0) return false;
        colour[i] = c;
        ncol = std::max(ncol, c + 1);
        for (int32_t k = inc_off[i]; k < inc_off[i + 1]; ++k)
            used[(size_t)inc_tet[k] * words + (c >> 6)] |= 1ull << (c & 63);
    }
    return true;
}

// Section "Collision Coloring": starting from the current colours, every
// free vertex of a weak constraint (ascending id) keeps its colour unless a
// vertex it shares a tet or a constraint with uses it, else takes the least
// colour none of them uses.  Vertices of constraints that were already there
// keep their colours, so only those of new constraints change.
void recolour_constraint_vertices(const pbng_mesh& m, const std::vector<int32_t>& inc_off,
                                  const std::vector<int32_t>& inc_tet, const std::vector<int32_t>& vwc_off,
                                  const std::vector<int32_t>& vwc, std::vector<int32_t>& colour, int32_t& ncol) {
    std::vector<uint8_t> used;
    for (int32_t i = 0; i < m.nv; ++i) {
        if (m.is_dir[i] || vwc_off[i + 1] == vwc_off[i]) continue;
        used.assign((size_t)ncol + 1, 0);
        auto mark = [&](int32_t v) {
            if (v != i && colour[v] >= 0) used[colour[v]] = 1;
        };
        for (int32_t k = inc_off[i]; k < inc_off[i + 1]; ++k)
            for (int j = 0; j < 4; ++j) mark(m.tets[4 * (size_t)inc_tet[k] + j]);
        for (int32_t k = vwc_off[i]; k < vwc_off[i + 1]; ++k)
            for (int32_t v : m.wc_v[vwc[k]]) mark(v);
        if (colour[i] >= 0 && !used[colour[i]]) continue;
        int32_t c = 0;
        while (used[c]) ++c;
        colour[i] = c;
        ncol = std::max(ncol, c + 1);
    }
}

int width_for(int deg) {
    if (deg <= 4) return 4;
    if (deg <= 8) return 8;
    if (deg <= 16) return 16;
    return 32;
}

// Builds the colour-ordered layout and uploads it.
//
// Internal vertex order: free vertices by colour, inside a colour by lane
// width (widest first) then caller id; clamped vertices last.  A vertex's
// lane width W is the smallest power of two (>= 4) holding both its incident
// tets and its 1-ring.  Colours whose vertices all have W <= 32 use the ring
// layout (pbng_ring.cu) unless direct loads were requested; the others use
// CSR records with direct loads (pbng_kernels.cu).
pbng_status build_layout(pbng_mesh* m) {
    const int32_t nv = m->nv, ne = m->ne;
    // vertex -> incident (tet, local) in ascending tet order
    std::vector<int32_t> inc_off(nv + 1, 0), inc_tet(4 * (size_t)ne), inc_loc(4 * (size_t)ne);
    for (int32_t v : m->tets) inc_off[v + 1]++;
    for (int32_t i = 0; i < nv; ++i) inc_off[i + 1] += inc_off[i];
    {
        std::vector<int32_t> fill(inc_off.begin(), inc_off.end() - 1);
        for (int32_t e = 0; e < ne; ++e)
            for (int j = 0; j < 4; ++j) {
                int32_t v = m->tets[4 * (size_t)e + j];
                inc_tet[fill[v]] = e;
                inc_loc[fill[v]] = j;
                fill[v]++;
            }
    }
    const auto t_start = std::chrono::steady_clock::now();
    // vertex -> weak constraints
    const int32_t nwc = (int32_t)m->wc_v.size();
    std::vector<int32_t> vwc_off(nv + 1, 0), vwc;
    for (const auto& c : m->wc_v)
        for (int32_t v : c) vwc_off[v + 1]++;
    for (int32_t i = 0; i < nv; ++i) vwc_off[i + 1] += vwc_off[i];
    vwc.resize(vwc_off[nv]);
    {
        std::vector<int32_t> fill(vwc_off.begin(), vwc_off.end() - 1);
        for (int32_t c = 0; c < nwc; ++c)
            for (int32_t v : m->wc_v[c]) vwc[fill[v]++] = c;
    }
    bool incremental = m->wc_incremental && (int32_t)m->colour.size() == nv;
    if (incremental)
        for (int32_t i = 0; i < nv && incremental; ++i) incremental = m->is_dir[i] || m->colour[i] >= 0;
    if (incremental) {
        int32_t ncol = 0;
        for (int32_t i = 0; i < nv; ++i) {
            if (m->is_dir[i]) m->colour[i] = -1;
            ncol = std::max(ncol, m->colour[i] + 1);
        }
        recolour_constraint_vertices(*m, inc_off, inc_tet, vwc_off, vwc, m->colour, ncol);
        m->ncol = ncol;
    } else {
        // tets and weak constraints are the elements of the greedy colouring
        std::vector<int32_t> ce_off(nv + 1, 0), ce;
        ce.reserve(inc_tet.size() + vwc.size());
        for (int32_t i = 0; i < nv; ++i) {
            ce.insert(ce.end(), inc_tet.begin() + inc_off[i], inc_tet.begin() + inc_off[i + 1]);
            for (int32_t k = vwc_off[i]; k < vwc_off[i + 1]; ++k) ce.push_back(ne + vwc[k]);
            ce_off[i + 1] = (int32_t)ce.size();
        }
        int words = 1;
        while (!greedy_colour(*m, ce_off, ce, ne + nwc, words, m->colour, m->ncol)) {
            words *= 2;
            if (words > 64) return fail(m, PBNG_EINVAL, "colouring needs more than 4096 colours");
        }
    }
    m->wc_incremental = false;
    m->colour_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    auto deg = [&](int32_t i) { return inc_off[i + 1] - inc_off[i]; };
    // 1-ring of each free vertex (caller ids, ascending)
    std::vector<int32_t> ring_off(nv + 1, 0), ring;
    {
        std::vector<int32_t> tmp;
        for (int32_t i = 0; i < nv; ++i) {
            if (!m->is_dir[i]) {
                tmp.clear();
                for (int32_t k = inc_off[i]; k < inc_off[i + 1]; ++k)
                    for (int j = 0; j < 4; ++j) {
                        const int32_t w = m->tets[4 * (size_t)inc_tet[k] + j];
                        if (w != i) tmp.push_back(w);
                    }
                std::sort(tmp.begin(), tmp.end());
                tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
                ring.insert(ring.end(), tmp.begin(), tmp.end());
            }
            ring_off[i + 1] = (int32_t)ring.size();
        }
    }
    auto ring_n = [&](int32_t i) { return ring_off[i + 1] - ring_off[i]; };
    auto lanes = [&](int32_t i) { return width_for(std::max(deg(i), ring_n(i))); };
    // pair items: two tets and two 1-ring vertices per lane
    auto lanes2 = [&](int32_t i) { return width_for(std::max((deg(i) + 1) / 2, (ring_n(i) + 1) / 2)); };

    std::vector<int32_t> order;
    order.reserve(nv);
    for (int32_t i = 0; i < nv; ++i)
        if (!m->is_dir[i]) order.push_back(i);
    // inside a colour and lane width, group the vertices of each component so
    // that most ring items hold a single component (and can be skipped whole
    // once that component has converged)
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (m->colour[a] != m->colour[b]) return m->colour[a] < m->colour[b];
        if (lanes(a) != lanes(b)) return lanes(a) > lanes(b);
        if (lanes2(a) != lanes2(b)) return lanes2(a) > lanes2(b);
        if (m->ncomp > 1 && m->comp_of[a] != m->comp_of[b]) return m->comp_of[a] < m->comp_of[b];
        return false;
    });
    m->nfree = (int32_t)order.size();
    for (int32_t i = 0; i < nv; ++i)
        if (m->is_dir[i]) order.push_back(i);
    m->perm = order;
    std::vector<int32_t> iperm(nv);
    for (int32_t v = 0; v < nv; ++v) iperm[order[v]] = v;

    // segments per colour, and which colours take the ring layout
    m->tables.assign(m->ncol, SegmentTable{});
    m->table_partial_off.assign(m->ncol + 1, 0);
    m->ring_colour.assign(m->ncol, 0);
    int32_t v = 0;
    for (int c = 0; c < m->ncol; ++c) {
        SegmentTable& t = m->tables[c];
        t.count = 0;
        t.total_blocks = 0;
        bool fits = true;
        while (v < m->nfree && m->colour[order[v]] == c) {
            const int W = lanes(order[v]);
            const int32_t b = v;
            while (v < m->nfree && m->colour[order[v]] == c && lanes(order[v]) == W) {
                if (std::max(deg(order[v]), ring_n(order[v])) > kRingLanes) fits = false;
                ++v;
            }
            if (t.count >= kMaxSegments) return fail(m, PBNG_EINVAL, "too many lane-width runs in a colour");
            Segment& sg = t.seg[t.count++];
            sg.v_begin = b;
            sg.v_end = v;
            sg.width = W;
            sg.block_begin = t.total_blocks;
            const int per_block = kBlock / W;
            t.total_blocks += (v - b + per_block - 1) / per_block;
        }
        m->ring_colour[c] = (fits && !m->want_direct) ? 1 : 0;
    }
    if ((int)m->sched.size() != m->ncol) {
        m->sched.assign(m->ncol, RingSched{ring_max_ctas_per_sm(), 0, 0});
        m->tune_default_ms = m->tune_ms = 0.0;
        m->tune_cands = 0;
    }
    m->all_ring = true;
    int32_t direct_partials = 0;
    for (int c = 0; c < m->ncol; ++c) {
        m->table_partial_off[c] = direct_partials;
        if (!m->ring_colour[c]) {
            m->all_ring = false;
            direct_partials += m->tables[c].total_blocks;
        }
    }
    m->table_partial_off[m->ncol] = direct_partials;
    m->total_partials = direct_partials;

    int64_t ninc_all = 0;
    for (int32_t w = 0; w < m->nfree; ++w) ninc_all += deg(order[w]);
    m->ninc = ninc_all;

    // CSR records for the direct-load colours (empty ranges elsewhere)
    std::vector<int32_t> off(m->nfree + 1, 0);
    for (int32_t w = 0; w < m->nfree; ++w)
        off[w + 1] = off[w] + (m->ring_colour[m->colour[order[w]]] ? 0 : deg(order[w]));
    const size_t ninc = (size_t)off[m->nfree];
    std::vector<float4> ra(ninc), rb(ninc), rc(ninc);
    std::vector<float2> rd(ninc);
    auto grads = [&](int32_t e, double g[4][3]) {
        const double* Be = &m->B[9 * (size_t)e];
        for (int a = 0; a < 3; ++a) {
            g[1][a] = Be[a];
            g[2][a] = Be[3 + a];
            g[3][a] = Be[6 + a];
            g[0][a] = -(Be[a] + Be[3 + a] + Be[6 + a]);
        }
    };
    for (int32_t w = 0; w < m->nfree; ++w) {
        const int32_t i = order[w];
        if (m->ring_colour[m->colour[i]]) continue;
        size_t s = off[w];
        for (int32_t k = inc_off[i]; k < inc_off[i + 1]; ++k, ++s) {
            const int32_t e = inc_tet[k];
            const int loc = inc_loc[k];
            double g[4][3];
            grads(e, g);
            int oth[3], n = 0;
            for (int j = 0; j < 4; ++j)
                if (j != loc) oth[n++] = j;
            int32_t ids[3];
            for (int q = 0; q < 3; ++q) ids[q] = iperm[m->tets[4 * (size_t)e + oth[q]]];
            float4 A4;
            std::memcpy(&A4.x, &ids[0], 4);
            std::memcpy(&A4.y, &ids[1], 4);
            std::memcpy(&A4.z, &ids[2], 4);
            A4.w = (float)(2.0 * m->mu[e] * m->vol[e]);
            ra[s] = A4;
            rb[s] = make_float4((float)g[oth[0]][0], (float)g[oth[0]][1], (float)g[oth[0]][2],
                                (float)(m->lam[e] * m->vol[e]));
            rc[s] = make_float4((float)g[oth[1]][0], (float)g[oth[1]][1], (float)g[oth[1]][2], (float)g[oth[2]][0]);
            rd[s] = make_float2((float)g[oth[2]][1], (float)g[oth[2]][2]);
        }
    }

    // ring layout: per lane-width run, 32-slot aligned; W slots per vertex
    m->items.clear();
    m->item_off.assign(m->ncol + 1, 0);
    std::vector<float4> qa, qb, qc, la, lb, lc;  // records and their low words
    std::vector<int32_t> qid;
    auto lo = [](double x) { return (float)(x - (double)(float)x); };
    for (int c = 0; c < m->ncol; ++c) {
        if (m->ring_colour[c]) {
            const SegmentTable& t = m->tables[c];
            for (int k = 0; k < t.count; ++k) {
                const Segment& sg = t.seg[k];
                const int W = sg.width;
                const int32_t slot_base = (int32_t)qa.size();  // a multiple of 32
                const int32_t nslots = ((sg.v_end - sg.v_begin) * W + kRingLanes - 1) / kRingLanes * kRingLanes;
                qa.resize(slot_base + nslots, make_float4(0.f, 0.f, 0.f, 0.f));
                qb.resize(slot_base + nslots, make_float4(0.f, 0.f, 0.f, 0.f));
                qc.resize(slot_base + nslots, make_float4(0.f, 0.f, 0.f, 0.f));
                la.resize(slot_base + nslots, make_float4(0.f, 0.f, 0.f, 0.f));
                lb.resize(slot_base + nslots, make_float4(0.f, 0.f, 0.f, 0.f));
                lc.resize(slot_base + nslots, make_float4(0.f, 0.f, 0.f, 0.f));
                qid.resize(slot_base + nslots, 0);
                for (int32_t vv = sg.v_begin; vv < sg.v_end; ++vv) {
                    const int32_t i = order[vv];
                    const int32_t s0 = slot_base + (vv - sg.v_begin) * W;
                    const int32_t* rg = &ring[ring_off[i]];
                    const int rn = ring_n(i);
                    for (int l = 0; l < W; ++l) qid[s0 + l] = l < rn ? iperm[rg[l]] : vv;
                    for (int32_t k2 = inc_off[i]; k2 < inc_off[i + 1]; ++k2) {
                        const int32_t slot = s0 + (k2 - inc_off[i]);
                        const int32_t e = inc_tet[k2];
                        const int loc = inc_loc[k2];
                        double g[4][3];
                        grads(e, g);
                        int oth[3], n = 0;
                        for (int j = 0; j < 4; ++j)
                            if (j != loc) oth[n++] = j;
                        int32_t packed = 0;
                        for (int q = 0; q < 3; ++q) {
                            const int32_t w = m->tets[4 * (size_t)e + oth[q]];
                            const int32_t l = (int32_t)(std::lower_bound(rg, rg + rn, w) - rg);
                            packed |= l << (8 * q);
                        }
                        float pk;
                        std::memcpy(&pk, &packed, 4);
                        qa[slot] = make_float4((float)g[oth[0]][0], (float)g[oth[0]][1], (float)g[oth[0]][2],
                                               (float)(2.0 * m->mu[e] * m->vol[e]));
                        qb[slot] = make_float4((float)g[oth[1]][0], (float)g[oth[1]][1], (float)g[oth[1]][2],
                                               (float)(m->lam[e] * m->vol[e]));
                        qc[slot] = make_float4((float)g[oth[2]][0], (float)g[oth[2]][1], (float)g[oth[2]][2], pk);
                        la[slot] = make_float4(lo(g[oth[0]][0]), lo(g[oth[0]][1]), lo(g[oth[0]][2]),
                                               lo(2.0 * m->mu[e] * m->vol[e]));
                        lb[slot] = make_float4(lo(g[oth[1]][0]), lo(g[oth[1]][1]), lo(g[oth[1]][2]),
                                               lo(m->lam[e] * m->vol[e]));
                        lc[slot] = make_float4(lo(g[oth[2]][0]), lo(g[oth[2]][1]), lo(g[oth[2]][2]), 0.f);
                    }
                }
                const int per_item = kRingLanes / W;
                for (int32_t vv = sg.v_begin; vv < sg.v_end; vv += per_item) {
                    Item it{};
                    it.v0 = vv;
                    it.nv = std::min<int32_t>(per_item, sg.v_end - vv);
                    it.w = W;
                    it.slot0 = slot_base + (vv - sg.v_begin) * W;
                    it.comp = m->ncomp > 1 ? m->comp_of[order[vv]] : 0;
                    for (int32_t q = 1; q < it.nv; ++q)
                        if (m->ncomp > 1 && m->comp_of[order[vv + q]] != it.comp) it.comp = -1;
                    m->items.push_back(it);
                }
            }
        }
        m->item_off[c + 1] = (int32_t)m->items.size();
    }
    m->nitems_ring = (int32_t)m->items.size();

    // pair layout of the same colours: per run of equal pair width W2 inside
    // a lane-width run, items of 32 / W2 vertices, one PairRec and one
    // PairIds each; lane l of a vertex's group holds its 1-ring vertices l and
    // W2 + l and its tets l and W2 + l
    m->pitems.clear();
    m->pitem_off.assign(m->ncol + 1, 0);
    std::vector<PairRec> precs;
    std::vector<PairIds> pids;
    for (int c = 0; c < m->ncol; ++c) {
        if (m->ring_colour[c]) {
            const SegmentTable& t = m->tables[c];
            for (int k = 0; k < t.count; ++k) {
                const Segment& sg = t.seg[k];
                for (int32_t rb = sg.v_begin; rb < sg.v_end;) {
                    const int W2 = lanes2(order[rb]);
                    // the pair kernel handles widths 4, 8 and 16 only
                    if (W2 > kRingLanes / 2) return fail(m, PBNG_EINVAL, "pair item wider than 16 lanes");
                    int32_t re = rb;
                    while (re < sg.v_end && lanes2(order[re]) == W2) ++re;
                    const int per_item = kRingLanes / W2;
                    for (int32_t vv = rb; vv < re; vv += per_item) {
                        Item it{};
                        it.v0 = vv;
                        it.nv = std::min<int32_t>(per_item, re - vv);
                        it.w = W2;
                        it.slot0 = (int32_t)precs.size() * kRingLanes;
                        it.comp = m->ncomp > 1 ? m->comp_of[order[vv]] : 0;
                        for (int32_t q = 1; q < it.nv; ++q)
                            if (m->ncomp > 1 && m->comp_of[order[vv + q]] != it.comp) it.comp = -1;
                        m->pitems.push_back(it);
                        PairRec rec;
                        PairIds ids;
                        std::memset(&rec, 0, sizeof(rec));
                        std::memset(&ids, 0, sizeof(ids));
                        float* val = reinterpret_cast<float*>(rec.r);
                        // value k2 of tet `tet` (0 = A, 1 = B) of lane `lane`
                        auto put = [&](int lane, int tet, int k2, float x) {
                            val[(k2 / 2) * 4 * kRingLanes + 4 * lane + 2 * (k2 % 2) + tet] = x;
                        };
                        for (int q = 0; q < it.nv; ++q) {
                            const int32_t w = vv + q;
                            const int32_t i = order[w];
                            const int32_t* rg = &ring[ring_off[i]];
                            const int rn = ring_n(i);
                            for (int l = 0; l < 2 * W2; ++l) ids.id[l / W2][q * W2 + l % W2] = l < rn ? iperm[rg[l]] : w;
                            for (int32_t k2 = inc_off[i]; k2 < inc_off[i + 1]; ++k2) {
                                const int slot = k2 - inc_off[i];
                                const int lane = q * W2 + slot % W2, tet = slot / W2;
                                const int32_t e = inc_tet[k2];
                                const int loc = inc_loc[k2];
                                double g[4][3];
                                grads(e, g);
                                int oth[3], n = 0;
                                for (int j = 0; j < 4; ++j)
                                    if (j != loc) oth[n++] = j;
                                // slots relative to the group's first lane
                                int32_t packed = 0;
                                for (int qq = 0; qq < 3; ++qq) {
                                    const int32_t w2 = m->tets[4 * (size_t)e + oth[qq]];
                                    const int32_t l = (int32_t)(std::lower_bound(rg, rg + rn, w2) - rg);
                                    packed |= ((l / W2) * kRingLanes + l % W2) << (8 * qq);
                                }
                                float pk;
                                std::memcpy(&pk, &packed, 4);
                                for (int jj = 0; jj < 3; ++jj)
                                    for (int a = 0; a < 3; ++a) put(lane, tet, 3 * jj + a, (float)g[oth[jj]][a]);
                                put(lane, tet, 9, (float)(2.0 * m->mu[e] * m->vol[e]));
                                put(lane, tet, 10, (float)(m->lam[e] * m->vol[e]));
                                put(lane, tet, 11, pk);
                            }
                        }
                        precs.push_back(rec);
                        pids.push_back(ids);
                    }
                    rb = re;
                }
            }
        }
        m->pitem_off[c + 1] = (int32_t)m->pitems.size();
    }
    m->nitems_pair = (int32_t)m->pitems.size();

    std::vector<float4> aux0(m->nfree), aux1(m->nfree), auxlo(m->nfree);
    std::vector<int32_t> comp(m->ncomp > 1 ? m->nfree : 0);
    for (int32_t w = 0; w < m->nfree; ++w) {
        const int32_t i = order[w];
        const double K = m->spr_K[i];
        float4 a0 = make_float4((float)m->fext[3 * i], (float)m->fext[3 * i + 1], (float)m->fext[3 * i + 2], (float)K);
        auxlo[w] = make_float4((float)(m->fext[3 * i] - (double)a0.x), (float)(m->fext[3 * i + 1] - (double)a0.y),
                               (float)(m->fext[3 * i + 2] - (double)a0.z), 0.f);
        float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (K > 0.0)
            for (int a = 0; a < 3; ++a)
                (&a1.x)[a] = (float)(m->spr_KT[3 * i + a] / K - m->X[3 * i + a]);
        if (m->has_plane)
            a1.w = (float)(m->pn[0] * m->X[3 * i] + m->pn[1] * m->X[3 * i + 1] + m->pn[2] * m->X[3 * i + 2] - m->pd);
        aux0[w] = a0;
        aux1[w] = a1;
        if (m->ncomp > 1) comp[w] = m->comp_of[i];
    }
    // Backward Euler: the inertia is a zero-rest spring of stiffness
    // m_i / dt^2 to the inertial target, which pbng_step sets; until then the
    // target is the rest position.
    std::vector<float4> base0, base1;
    std::vector<float> bek;
    if (m->be_dt > 0.0) {
        base0 = aux0;
        base1 = aux1;
        bek.resize(m->nfree);
        for (int32_t w = 0; w < m->nfree; ++w) {
            const double k = m->be_mass[order[w]] / (m->be_dt * m->be_dt);
            const double Ks = aux0[w].w, K = Ks + k;
            bek[w] = (float)k;
            aux0[w].w = (float)K;
            for (int a = 0; a < 3; ++a) (&aux1[w].x)[a] = (float)(Ks * (&base1[w].x)[a] / K);
        }
    }
    const int32_t nd = nv - m->nfree;
    std::vector<float4> dhi(nd), dlo(nd);
    for (int32_t q = 0; q < nd; ++q) {
        const int32_t i = order[m->nfree + q];
        float h[3], l[3];
        for (int a = 0; a < 3; ++a) {
            const double d = m->dir_pos[3 * i + a] - m->X[3 * i + a];
            h[a] = (float)d;
            l[a] = (float)(d - (double)h[a]);
        }
        dhi[q] = make_float4(h[0], h[1], h[2], 0.f);
        dlo[q] = make_float4(l[0], l[1], l[2], 0.f);
    }
    cudaStream_t st = m->stream;
    PBNG_CUDA(m, upload(m->d_inc_off, off, st));
    PBNG_CUDA(m, upload(m->d_rec_a, ra, st));
    PBNG_CUDA(m, upload(m->d_rec_b, rb, st));
    PBNG_CUDA(m, upload(m->d_rec_c, rc, st));
    PBNG_CUDA(m, upload(m->d_rec_d, rd, st));
    {
        std::vector<RingBlock> blocks(qa.size() / kRingLanes);
        for (size_t q = 0; q < qa.size(); ++q) {
            RingBlock& b = blocks[q / kRingLanes];
            b.ra[q % kRingLanes] = qa[q];
            b.rb[q % kRingLanes] = qb[q];
            b.rc[q % kRingLanes] = qc[q];
            b.id[q % kRingLanes] = qid[q];
        }
        PBNG_CUDA(m, upload(m->d_ring, blocks, st));
        std::vector<RingLoBlock> lblocks(la.size() / kRingLanes);
        for (size_t q = 0; q < la.size(); ++q) {
            RingLoBlock& b = lblocks[q / kRingLanes];
            b.la[q % kRingLanes] = la[q];
            b.lb[q % kRingLanes] = lb[q];
            b.lc[q % kRingLanes] = lc[q];
        }
        PBNG_CUDA(m, upload(m->d_ring_lo, lblocks, st));
    }
    PBNG_CUDA(m, upload(m->d_items, m->items, st));
    PBNG_CUDA(m, upload(m->d_prec, precs, st));
    PBNG_CUDA(m, upload(m->d_pids, pids, st));
    PBNG_CUDA(m, upload(m->d_pitems, m->pitems, st));
    PBNG_CUDA(m, upload(m->d_aux0, aux0, st));
    PBNG_CUDA(m, upload(m->d_aux1, aux1, st));
    PBNG_CUDA(m, upload(m->d_aux_lo, auxlo, st));
    if (m->be_dt > 0.0) {
        PBNG_CUDA(m, upload(m->d_aux_base0, base0, st));
        PBNG_CUDA(m, upload(m->d_aux_base1, base1, st));
        PBNG_CUDA(m, upload(m->d_be_k, bek, st));
    }
    if (nwc > 0) {
        // constraint tables in internal ids; per free vertex, its constraints
        std::vector<int32_t> iperm(nv);
        for (int32_t w = 0; w < nv; ++w) iperm[order[w]] = w;
        std::vector<int32_t> cv(8 * (size_t)nwc, -1);
        std::vector<float> cb(8 * (size_t)nwc, 0.f), ck(6 * (size_t)nwc);
        std::vector<float4> c0(2 * (size_t)nwc);
        for (int32_t c = 0; c < nwc; ++c) {
            double C0[3] = {0.0, 0.0, 0.0};
            for (size_t q = 0; q < m->wc_v[c].size(); ++q) {
                const int32_t v = m->wc_v[c][q];
                cv[8 * (size_t)c + q] = iperm[v];
                cb[8 * (size_t)c + q] = (float)m->wc_b[c][q];
                for (int a = 0; a < 3; ++a) C0[a] += m->wc_b[c][q] * m->X[3 * (size_t)v + a];
            }
            for (int k = 0; k < 6; ++k) ck[6 * (size_t)c + k] = (float)m->wc_k[c][k];
            const float h0 = (float)C0[0], h1 = (float)C0[1], h2 = (float)C0[2];
            c0[2 * (size_t)c] = make_float4(h0, h1, h2, 0.f);
            c0[2 * (size_t)c + 1] = make_float4((float)(C0[0] - h0), (float)(C0[1] - h1), (float)(C0[2] - h2), 0.f);
        }
        std::vector<int32_t> woff(m->nfree + 1, 0);
        std::vector<int2> wlist;
        for (int32_t w = 0; w < m->nfree; ++w) {
            const int32_t i = order[w];
            for (int32_t k = vwc_off[i]; k < vwc_off[i + 1]; ++k) {
                const int32_t c = vwc[k];
                double b = 0.0;
                for (size_t q = 0; q < m->wc_v[c].size(); ++q)
                    if (m->wc_v[c][q] == i) b = m->wc_b[c][q];
                const float bf = (float)b;
                int32_t bits;
                std::memcpy(&bits, &bf, sizeof(bits));
                wlist.push_back(make_int2(c, bits));
            }
            woff[w + 1] = (int32_t)wlist.size();
        }
        PBNG_CUDA(m, upload(m->d_wc_off, woff, st));
        PBNG_CUDA(m, upload(m->d_wc_list, wlist, st));
        PBNG_CUDA(m, upload(m->d_wc_v, cv, st));
        PBNG_CUDA(m, upload(m->d_wc_b, cb, st));
        PBNG_CUDA(m, upload(m->d_wc_k, ck, st));
        PBNG_CUDA(m, upload(m->d_wc_c0, c0, st));
    }
    PBNG_CUDA(m, upload(m->d_comp, comp, st));
    if (m->ncomp > 1) {  // component -> its free vertices (internal ids, ascending)
        std::vector<int32_t> coff(m->ncomp + 1, 0), clist(m->nfree);
        for (int32_t w = 0; w < m->nfree; ++w) coff[comp[w] + 1]++;
        for (int32_t k = 0; k < m->ncomp; ++k) coff[k + 1] += coff[k];
        std::vector<int32_t> fill(coff.begin(), coff.end() - 1);
        for (int32_t w = 0; w < m->nfree; ++w) clist[fill[comp[w]]++] = w;
        PBNG_CUDA(m, upload(m->d_comp_off, coff, st));
        PBNG_CUDA(m, upload(m->d_comp_list, clist, st));
        PBNG_CUDA(m, ensure_buf(m->d_vsq, sizeof(double) * (size_t)std::max(1, m->nfree)));
    }
    PBNG_CUDA(m, upload(m->d_perm, m->perm, st));
    PBNG_CUDA(m, upload(m->d_dir_hi, dhi, st));
    PBNG_CUDA(m, upload(m->d_dir_lo, dlo, st));
    for (auto& sb : m->d_state)
        for (auto& b : sb) PBNG_CUDA(m, ensure_buf(b, sizeof(float4) * (size_t)nv));
    destroy_graphs(m);
    PBNG_CUDA(m, ring_prepare());
    PBNG_CUDA(m, adjoint_prepare());
    PBNG_CUDA(m, ensure_buf(m->d_wg, sizeof(float2) * kMaxChunk));
    m->ring_partials = ring_warps(std::max(m->nitems_ring, m->nitems_pair));
    PBNG_CUDA(m, ensure_buf(m->d_partial, sizeof(double) * (size_t)std::max(1, m->ring_partials + m->total_partials)));
    PBNG_CUDA(m, ensure_buf(m->d_comp_sq, sizeof(double) * (size_t)m->ncomp));
    PBNG_CUDA(m, ensure_buf(m->d_active, sizeof(int32_t) * (size_t)m->ncomp));
    for (int32_t k = 0; k < m->ncomp; ++k) m->h_active[k] = 1;
    PBNG_CUDA(m, cudaMemcpyAsync(m->d_active.p, m->h_active, sizeof(int32_t) * m->ncomp,
                                 cudaMemcpyHostToDevice, st));
    PBNG_CUDA(m, cudaStreamSynchronize(st));
    PBNG_CUDA(m, ensure_buf(m->d_scalar, sizeof(double) * 4));
    PBNG_CUDA(m, ensure_buf(m->d_err, sizeof(int32_t)));
    PBNG_CUDA(m, cudaMemsetAsync(m->d_err.p, 0, sizeof(int32_t), st));

    DeviceMesh& d = m->dm;
    d.nv = nv;
    d.nfree = m->nfree;
    d.inc_off = (const int32_t*)m->d_inc_off.p;
    d.rec_a = (const float4*)m->d_rec_a.p;
    d.rec_b = (const float4*)m->d_rec_b.p;
    d.rec_c = (const float4*)m->d_rec_c.p;
    d.rec_d = (const float2*)m->d_rec_d.p;
    d.aux0 = (const float4*)m->d_aux0.p;
    d.aux1 = (const float4*)m->d_aux1.p;
    d.aux_lo = (const float4*)m->d_aux_lo.p;
    d.comp = m->ncomp > 1 ? (const int32_t*)m->d_comp.p : nullptr;
    d.comp_active = m->ncomp > 1 ? (const int32_t*)m->d_active.p : nullptr;
    d.vsq = m->ncomp > 1 ? (double*)m->d_vsq.p : nullptr;
    d.ring = (const RingBlock*)m->d_ring.p;
    d.ring_lo = (const RingLoBlock*)m->d_ring_lo.p;
    d.prec = (const PairRec*)m->d_prec.p;
    d.pids = (const PairIds*)m->d_pids.p;
    d.copy_shortfall = m->copy_shortfall;
    d.pn_x = (float)m->pn[0];
    d.pn_y = (float)m->pn[1];
    d.pn_z = (float)m->pn[2];
    d.k_contact = m->has_plane ? (float)m->kc : 0.0f;
    const bool has_wc = !m->wc_v.empty();
    d.wc_off = has_wc ? (const int32_t*)m->d_wc_off.p : nullptr;
    d.wc_list = has_wc ? (const int2*)m->d_wc_list.p : nullptr;
    d.wc_v = has_wc ? (const int32_t*)m->d_wc_v.p : nullptr;
    d.wc_b = has_wc ? (const float*)m->d_wc_b.p : nullptr;
    d.wc_k = has_wc ? (const float*)m->d_wc_k.p : nullptr;
    d.wc_c0 = has_wc ? (const float4*)m->d_wc_c0.p : nullptr;
    m->layout_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    m->built_direct = m->want_direct;
    m->adj_ready = false;
    m->dirty = false;
    m->has_state = false;
    return PBNG_OK;
}

State state_of(pbng_mesh* m, int slot) {
    return State{(float4*)m->d_state[slot][0].p, (float4*)m->d_state[slot][1].p};
}

pbng_status ensure_ready(pbng_mesh* m) {
    if (!m) return PBNG_EINVAL;
    m->err.clear();
    cudaError_t e = cudaSetDevice(m->device);
    if (e != cudaSuccess) return cuda_fail(m, e, "cudaSetDevice");
    if (m->dirty) return build_layout(m);
    return PBNG_OK;
}

// Enqueues the FP64 squared residual norms of state `s`: the ring launch
// writes ring_partials per-warp partials at partial[0..), each direct-load
// colour its per-block partials after them; then the sum lands in *scalar.
// With several components the sums go to comp_sq (zeroed here) instead.
// extended: float-float element forces (every colour is in the ring layout).
// With several components each vertex's |r|^2 lands in its slot of d_vsq
// and the per-component sums follow in a fixed order (the same bits every
// run); atomic_comp (the allocation-free residual, which has no slots) sums
// them atomically into comp_sq instead.
pbng_status enqueue_residual(pbng_mesh* m, State s, bool compensated, double* partial, double* comp_sq,
                             double* scalar, cudaStream_t st, bool extended = false, bool atomic_comp = false) {
    const bool multi = m->ncomp > 1;
    DeviceMesh dm = m->dm;
    if (multi && atomic_comp) {
        dm.vsq = nullptr;
        PBNG_CUDA(m, cudaMemsetAsync(comp_sq, 0, sizeof(double) * m->ncomp, st));
    } else if (multi) {  // vertices of frozen items are not written: they count as zero
        PBNG_CUDA(m, cudaMemsetAsync(m->d_vsq.p, 0, sizeof(double) * (size_t)m->nfree, st));
    }
    if (m->nitems_ring > 0) {
        const bool ext = extended && compensated;
        PBNG_CUDA(m, launch_ring_residual(dm, s, (const Item*)(ext ? m->d_items.p : m->d_pitems.p),
                                          ext ? m->nitems_ring : m->nitems_pair, compensated, partial,
                                          multi ? comp_sq : nullptr, m->model, (int32_t*)m->d_err.p, st, ext,
                                          m->ring_partials));
        m->kernel_launches++;
    }
    for (int c = 0; c < m->ncol; ++c) {
        if (m->ring_colour[c]) continue;
        PBNG_CUDA(m, launch_residual(dm, s, m->tables[c], compensated,
                                     partial + m->ring_partials + m->table_partial_off[c],
                                     multi ? comp_sq : nullptr, m->ncomp, nullptr, m->model, st));
        if (m->tables[c].total_blocks > 0) m->kernel_launches++;
    }
    if (!multi) {
        PBNG_CUDA(m, launch_reduce(partial, m->ring_partials + m->total_partials, scalar, st));
        m->kernel_launches++;
    } else if (!atomic_comp) {
        PBNG_CUDA(m, launch_comp_reduce(m->ncomp, (const int32_t*)m->d_comp_off.p, (const int32_t*)m->d_comp_list.p,
                                        (const double*)m->d_vsq.p, comp_sq, st));
        m->kernel_launches++;
    }
    return PBNG_OK;
}

pbng_status sync_with_err(pbng_mesh* m, cudaStream_t st);

// FP64 squared residual norms (per component) of state `slot` -> host `out`.
pbng_status residual_sq(pbng_mesh* m, int slot, bool compensated, double* out, bool extended = false) {
    cudaStream_t st = m->stream;
    const bool multi = m->ncomp > 1;
    const int pslot = prof_begin(m, kProfResidual);
    pbng_status r = enqueue_residual(m, state_of(m, slot), compensated, (double*)m->d_partial.p,
                                     (double*)m->d_comp_sq.p, (double*)m->d_scalar.p, st, extended);
    if (r) return r;
    prof_end(m, pslot);
    PBNG_CUDA(m, cudaMemcpyAsync(m->h_pinned, multi ? m->d_comp_sq.p : m->d_scalar.p,
                                 sizeof(double) * (multi ? m->ncomp : 1), cudaMemcpyDeviceToHost, st));
    if ((r = sync_with_err(m, st))) return r;  // a timed-out warp left its partial at zero
    for (int k = 0; k < m->ncomp; ++k) out[k] = (m->ncol == 0) ? 0.0 : m->h_pinned[k];
    return PBNG_OK;
}

pbng_status check_err(pbng_mesh* m) {
    int32_t h = 0;
    PBNG_CUDA(m, cudaMemcpyAsync(&h, m->d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream));
    PBNG_CUDA(m, cudaStreamSynchronize(m->stream));
    if (h) {
        PBNG_CUDA(m, cudaMemsetAsync(m->d_err.p, 0, sizeof(int32_t), m->stream));
        if (h & kErrTimeout) return fail(m, PBNG_ETIMEOUT, "asynchronous copy wait gave up");
        if (h & kErrNonSPD) return fail(m, PBNG_EDEGENERATE, "nodal Hessian not positive definite");
        return fail(m, PBNG_EDIVERGED, "non-finite vertex update");
    }
    return PBNG_OK;
}

// Synchronises the stream after also reading the device error flag into the
// spare pinned slot after the per-component readbacks, and reports a set
// flag (which check_err then clears): one synchronisation for both.
pbng_status sync_with_err(pbng_mesh* m, cudaStream_t st) {
    int32_t* herr = reinterpret_cast<int32_t*>(m->h_pinned + m->ncomp);
    *herr = 0;
    PBNG_CUDA(m, cudaMemcpyAsync(herr, m->d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PBNG_CUDA(m, cudaStreamSynchronize(st));
    return *herr ? check_err(m) : PBNG_OK;
}

// kernel_path 1 (direct loads everywhere) needs CSR records for every
// colour: switching path rebuilds the layout (and drops the iterate history).
void select_path(pbng_mesh* m, const pbng_params* p) {
    m->model = p->model;
    m->want_direct = p->kernel_path == 1;
    if (m->want_direct != m->built_direct) m->dirty = true;
}

bool valid_params(const pbng_params* p) {
    return p && p->model >= 0 && p->model <= 2 && p->accel >= 0 && p->accel <= 2 && p->residual_every >= 1 &&
           p->precision >= PBNG_PREC_FP32 && p->precision <= PBNG_PREC_AUTO &&
           std::isfinite(p->omega) && std::isfinite(p->rho) && std::isfinite(p->gamma) &&
           std::isfinite(p->step) && p->skip_tol >= 0.0 && (p->kernel_path == 0 || p->kernel_path == 1) &&
           (p->colour_order == PBNG_ORDER_FORWARD || p->colour_order == PBNG_ORDER_SYMMETRIC);
}

// Precision modes: the iterate is a float pair unless FP32; colour passes,
// and the residual checks inside a chunk of sweeps, use the float-float
// element force only in EXTENDED; the reported residuals (r_0, the final
// residual of pbng_sweep / pbng_sweep_host, the confirmation of a converged
// AUTO solve) use it in EXTENDED and AUTO.  pbng_solve moves AUTO's passes
// to EXTENDED when its checks stall.
bool pair_iterate(int prec) { return prec != PBNG_PREC_FP32; }
bool ext_passes(int prec) { return prec == PBNG_PREC_EXTENDED; }
bool ext_residual(int prec) { return prec == PBNG_PREC_EXTENDED || prec == PBNG_PREC_AUTO; }

// Extended-precision passes and residuals run on the ring layout only.
pbng_status check_ext(pbng_mesh* m, const pbng_params* p) {
    if ((ext_passes(p->precision) || ext_residual(p->precision)) && !m->all_ring)
        return fail(m, PBNG_EINVAL, "extended precision needs every colour in the ring layout (kernel_path 0)");
    return PBNG_OK;
}

// Colour passes of one sweep: 0..C-1, and for the symmetric order back down
// C-2..0 (the palindrome of symmetric Gauss-Seidel).
std::vector<int> colour_sequence(int ncol, int order) {
    std::vector<int> seq;
    for (int c = 0; c < ncol; ++c) seq.push_back(c);
    if (order == PBNG_ORDER_SYMMETRIC)
        for (int c = ncol - 2; c >= 0; --c) seq.push_back(c);
    return seq;
}

// Loads u_dev (or keeps the stored iterate) and resets the history.
pbng_status begin(pbng_mesh* m, const float* u_dev, const pbng_params* p, bool need_r0) {
    const bool comp = pair_iterate(p->precision);
    if (!p->resume || !m->has_state) {
        if (!u_dev) return fail(m, PBNG_EINVAL, "u_dev is NULL");
        PBNG_CUDA(m, launch_load(m->nv, m->nfree, u_dev, (const int32_t*)m->d_perm.p,
                                 (const float4*)m->d_dir_hi.p, (const float4*)m->d_dir_lo.p,
                                 state_of(m, 0), m->stream));
        PBNG_CUDA(m, launch_copy_state(m->nv, state_of(m, 0), state_of(m, 1), m->stream));
        PBNG_CUDA(m, launch_copy_state(m->nv, state_of(m, 0), state_of(m, 2), m->stream));
        m->kernel_launches += 3;
        m->p1_slot = 1;
        m->p2_slot = 2;
        m->sweep_l = 0;
        m->omega_l = 1.0;
        m->has_state = true;
        m->r0.assign(m->ncomp, -1.0);
    }
    if (need_r0 && (m->r0.empty() || m->r0[0] < 0.0)) {
        m->r0.assign(m->ncomp, 0.0);
        pbng_status s = residual_sq(m, 0, comp, m->r0.data(), ext_residual(p->precision));
        if (s) return s;
        for (auto& r : m->r0) r = std::sqrt(r);
    }
    return PBNG_OK;
}

// (w, g) of the acceleration step after each of the next K sweeps
// (Section "Acceleration Techniques"), advancing the host copy of the sweep
// index and of omega_l.  Chebyshev: omega_{l+1} = 1 (l < 2), 2/(2 - rho^2)
// (l = 2), 4/(4 - rho^2 omega_l) (l > 2), g = gamma.  SOR: (omega, 1).
void chunk_weights(pbng_mesh* m, const pbng_params* p, int32_t K, float2* out) {
    for (int32_t k = 0; k < K; ++k) {
        double w = 1.0, g = 1.0;
        const int l = m->sweep_l + k;
        if (p->accel == PBNG_ACCEL_CHEBYSHEV) {
            if (l < 2) w = 1.0;
            else if (l == 2) w = 2.0 / (2.0 - p->rho * p->rho);
            else w = 4.0 / (4.0 - p->rho * p->rho * m->omega_l);
            m->omega_l = w;
            g = p->gamma;
        } else if (p->accel == PBNG_ACCEL_SOR) {
            w = p->omega;
        }
        out[k] = make_float2((float)w, (float)g);
    }
    m->sweep_l += K;
}

// Enqueues K sweeps (every colour pass, then the acceleration step with the
// weights at d_wg[k]) and, with with_res, the FP64 residual and its copy to
// h_pinned.  Captured into a graph, or enqueued directly on the handle's
// stream when profiling.  p1 is the slot holding x^l at the start.
pbng_status enqueue_chunk(pbng_mesh* m, const pbng_params* p, int32_t K, bool with_res, int p1,
                          bool prof, int64_t* nkernels, cudaStream_t st) {
    const bool comp = pair_iterate(p->precision);
    const bool ext = ext_passes(p->precision);
    const PassParams pp{(float)p->step, (float)p->skip_tol, p->model};
    const State cur = state_of(m, 0);
    int p2 = 3 - p1;
    // With profiling (never inside a capture) each timed launch is bracketed
    // by a pair of pooled events.
    int slot = -1;
    auto mark = [&](int kind) -> pbng_status {
        if (!prof) return PBNG_OK;
        if (slot < 0) slot = prof_begin(m, kind);
        else { prof_end(m, slot); slot = -1; }
        return PBNG_OK;
    };
    pbng_status r;
    const std::vector<int> seq = colour_sequence(m->ncol, p->colour_order);
    for (int32_t k = 0; k < K; ++k) {
        for (const int c : seq) {
            if (m->tables[c].total_blocks <= 0) continue;
            if ((r = mark(kProfColour))) return r;
            if (m->ring_colour[c] && ext)
                PBNG_CUDA(m, launch_ring_pass(m->dm, cur, (const Item*)m->d_items.p + m->item_off[c],
                                              m->item_off[c + 1] - m->item_off[c], pp, comp, m->sched[c],
                                              (int32_t*)m->d_err.p, st, true));
            else if (m->ring_colour[c])
                PBNG_CUDA(m, launch_ring_pass(m->dm, cur, (const Item*)m->d_pitems.p + m->pitem_off[c],
                                              m->pitem_off[c + 1] - m->pitem_off[c], pp, comp, m->sched[c],
                                              (int32_t*)m->d_err.p, st));
            else
                PBNG_CUDA(m, launch_colour_pass(m->dm, cur, m->tables[c], pp, comp, (int32_t*)m->d_err.p, st));
            if ((r = mark(kProfColour))) return r;
            (*nkernels)++;
        }
        if (p->accel != PBNG_ACCEL_NONE && m->nfree > 0) {
            if ((r = mark(kProfAccel))) return r;
            PBNG_CUDA(m, launch_accel(m->nfree, cur, state_of(m, p1), state_of(m, p2),
                                      (const float2*)m->d_wg.p + k, m->dm.comp, m->dm.comp_active, comp, st));
            if ((r = mark(kProfAccel))) return r;
            (*nkernels)++;
            std::swap(p1, p2);
        }
    }
    if (with_res) {
        const bool multi = m->ncomp > 1;
        if ((r = mark(kProfResidual))) return r;
        const int64_t before = m->kernel_launches;
        if ((r = enqueue_residual(m, cur, comp, (double*)m->d_partial.p, (double*)m->d_comp_sq.p,
                                  (double*)m->d_scalar.p, st, ext)))
            return r;
        *nkernels += m->kernel_launches - before;
        m->kernel_launches = before;
        if ((r = mark(kProfResidual))) return r;
        PBNG_CUDA(m, cudaMemcpyAsync(m->h_pinned, multi ? m->d_comp_sq.p : m->d_scalar.p,
                                     sizeof(double) * (multi ? m->ncomp : 1), cudaMemcpyDeviceToHost, st));
    }
    return PBNG_OK;
}

// Runs K <= kMaxChunk sweeps (and the residual) as one CUDA graph launch,
// capturing the graph the first time a configuration is seen.  host_wg
// (pinned) must stay untouched until the stream reaches this chunk.
pbng_status run_chunk(pbng_mesh* m, const pbng_params* p, int32_t K, bool with_res, float2* host_wg) {
    cudaStream_t st = m->stream;
    chunk_weights(m, p, K, host_wg);
    PBNG_CUDA(m, cudaMemcpyAsync(m->d_wg.p, host_wg, sizeof(float2) * K, cudaMemcpyHostToDevice, st));
    const int32_t accel = (p->accel != PBNG_ACCEL_NONE && m->nfree > 0) ? 1 : 0;
    if (m->prof) {
        // per-launch timing needs plain launches (captured event records
        // cannot be timed): the same kernels, enqueued one by one
        int64_t nk = 0;
        pbng_status r = enqueue_chunk(m, p, K, with_res, m->p1_slot, true, &nk, st);
        if (r) return r;
        m->kernel_launches += nk;
        if (accel && (K & 1)) std::swap(m->p1_slot, m->p2_slot);
        return PBNG_OK;
    }
    pbng_mesh::GraphEntry* g = nullptr;
    for (auto& e : m->graphs)
        if (e.K == K && e.accel == accel && e.prec == p->precision && e.with_res == (int)with_res &&
            e.p1 == m->p1_slot && e.step == (float)p->step && e.skip == (float)p->skip_tol && e.model == p->model &&
            e.order == p->colour_order)
            g = &e;
    if (!g) {
        pbng_mesh::GraphEntry e;
        e.K = K;
        e.accel = accel;
        e.prec = p->precision;
        e.with_res = with_res;
        e.p1 = m->p1_slot;
        e.prof = 0;
        e.step = (float)p->step;
        e.skip = (float)p->skip_tol;
        e.model = p->model;
        e.order = p->colour_order;
        if (!m->cap_stream) PBNG_CUDA(m, cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        PBNG_CUDA(m, cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
        pbng_status r;
        {
            PdlScope pdl(true);  // each kernel of the chunk may start while its predecessor drains
            r = enqueue_chunk(m, p, K, with_res, m->p1_slot, false, &e.nkernels, m->cap_stream);
        }
        const cudaError_t ce = cudaStreamEndCapture(m->cap_stream, &graph);
        if (r) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (ce != cudaSuccess) return cuda_fail(m, ce, "cudaStreamEndCapture");
        const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_fail(m, ie, "cudaGraphInstantiate");
        m->graphs.push_back(std::move(e));
        g = &m->graphs.back();
    }
    PBNG_CUDA(m, cudaGraphLaunch(g->exec, st));
    m->kernel_launches += g->nkernels;
    if (accel && (K & 1)) std::swap(m->p1_slot, m->p2_slot);
    return PBNG_OK;
}

pbng_status ensure_wg(pbng_mesh* m, size_t n) {
    if (m->h_wg_cap >= n) return PBNG_OK;
    if (m->h_wg) cudaFreeHost(m->h_wg);
    m->h_wg = nullptr;
    m->h_wg_cap = 0;
    PBNG_CUDA(m, cudaMallocHost((void**)&m->h_wg, sizeof(float2) * n));
    m->h_wg_cap = n;
    return PBNG_OK;
}

}  // namespace

extern "C" {

void pbng_default_params(pbng_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->model = 0;
    p->accel = PBNG_ACCEL_NONE;
    p->omega = 1.7;
    p->rho = 0.95;
    p->gamma = 1.7;
    p->step = 1.0;
    p->skip_tol = 0.0;
    p->residual_every = 10;
    p->resume = 0;
    p->precision = PBNG_PREC_COMPENSATED;
}

pbng_status pbng_create_mesh(const double* rest_xyz, int32_t nv, const int32_t* tets, int32_t ne,
                             const double* young, const double* poisson, const int32_t* mesh_id,
                             void* stream, pbng_mesh** out) {
    if (!out) return PBNG_EINVAL;
    *out = nullptr;
    if (!rest_xyz || nv <= 0 || ne <= 0 || !tets || !young || !poisson) return PBNG_EINVAL;
    if ((int64_t)ne * 4 > INT32_MAX) return PBNG_EINVAL;
    pbng_mesh* m = new (std::nothrow) pbng_mesh();
    if (!m) return PBNG_ENOMEM;
    try {
        if (cudaGetDevice(&m->device) != cudaSuccess) { delete m; return PBNG_ECUDA; }
        m->stream = (cudaStream_t)stream;
        m->err.reserve(kErrTextReserve);
        m->nv = nv;
        m->ne = ne;
        m->X.assign(rest_xyz, rest_xyz + 3 * (size_t)nv);
        m->tets.assign(tets, tets + 4 * (size_t)ne);
        for (int32_t v : m->tets)
            if (v < 0 || v >= nv) { delete m; return PBNG_EINVAL; }
        m->B.resize(9 * (size_t)ne);
        m->vol.resize(ne);
        m->mu.resize(ne);
        m->lam.resize(ne);
        for (int32_t e = 0; e < ne; ++e) {
            const int32_t* t = &m->tets[4 * (size_t)e];
            double Dm[9], hmax = 0.0;
            for (int c = 0; c < 3; ++c)
                for (int a = 0; a < 3; ++a) {
                    Dm[3 * a + c] = m->X[3 * (size_t)t[c + 1] + a] - m->X[3 * (size_t)t[0] + a];
                    hmax = std::max(hmax, std::fabs(Dm[3 * a + c]));
                }
            const double D = det3(Dm);
            if (!(std::fabs(D) / 6.0 > 1e-12 * hmax * hmax * hmax)) { delete m; return PBNG_EDEGENERATE; }
            // rows of Dm^{-1} = columns of cof(Dm) / det
            const double C[9] = {Dm[4] * Dm[8] - Dm[5] * Dm[7], Dm[5] * Dm[6] - Dm[3] * Dm[8],
                                 Dm[3] * Dm[7] - Dm[4] * Dm[6], Dm[7] * Dm[2] - Dm[8] * Dm[1],
                                 Dm[8] * Dm[0] - Dm[6] * Dm[2], Dm[6] * Dm[1] - Dm[7] * Dm[0],
                                 Dm[1] * Dm[5] - Dm[2] * Dm[4], Dm[2] * Dm[3] - Dm[0] * Dm[5],
                                 Dm[0] * Dm[4] - Dm[1] * Dm[3]};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) m->B[9 * (size_t)e + 3 * a + b] = C[3 * b + a] / D;
            m->vol[e] = std::fabs(D) / 6.0;
            const double E = young[e], nu = poisson[e];
            if (!(E > 0.0) || !(nu >= 0.0 && nu < 0.5)) { delete m; return PBNG_EINVAL; }
            m->mu[e] = E / (2.0 * (1.0 + nu));                       // Eq. lame
            m->lam[e] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        }
        if (mesh_id) {
            m->comp_of.assign(mesh_id, mesh_id + nv);
            int32_t mx = -1;
            for (int32_t c : m->comp_of) {
                if (c < 0) { delete m; return PBNG_EINVAL; }
                mx = std::max(mx, c);
            }
            m->ncomp = mx + 1;
        }
        m->is_dir.assign(nv, 0);
        m->dir_pos.assign(3 * (size_t)nv, 0.0);
        m->spr_K.assign(nv, 0.0);
        m->spr_KT.assign(3 * (size_t)nv, 0.0);
        m->fext.assign(3 * (size_t)nv, 0.0);
        if (cudaMallocHost((void**)&m->h_pinned, sizeof(double) * (m->ncomp + 2)) != cudaSuccess ||
            cudaMallocHost((void**)&m->h_active, sizeof(int32_t) * m->ncomp) != cudaSuccess) {
            if (m->h_pinned) cudaFreeHost(m->h_pinned);
            delete m;
            return PBNG_ECUDA;
        }
    } catch (const std::bad_alloc&) {
        delete m;
        return PBNG_ENOMEM;
    }
    *out = m;
    return PBNG_OK;
}

pbng_status pbng_set_constraints(pbng_mesh* m, const int32_t* dir_idx, const double* dir_xyz,
                                 int32_t nd, const int32_t* spr_idx, const double* spr_target,
                                 const double* spr_k, int32_t ns, const double* plane_nd,
                                 double k_contact, const double* body_accel, const double* density) {
    if (!m) return PBNG_EINVAL;
    m->err.clear();
    if (nd < 0 || ns < 0 || (nd > 0 && (!dir_idx || !dir_xyz)) ||
        (ns > 0 && (!spr_idx || !spr_target || !spr_k)))
        return fail(m, PBNG_EINVAL, "bad constraint arrays");
    try {
        std::fill(m->is_dir.begin(), m->is_dir.end(), 0);
        m->dir_list.assign(dir_idx, dir_idx + nd);
        for (int32_t q = 0; q < nd; ++q) {
            const int32_t i = dir_idx[q];
            if (i < 0 || i >= m->nv) return fail(m, PBNG_EINVAL, "clamped id out of range");
            m->is_dir[i] = 1;
            for (int a = 0; a < 3; ++a) m->dir_pos[3 * (size_t)i + a] = dir_xyz[3 * (size_t)q + a];
        }
        std::fill(m->spr_K.begin(), m->spr_K.end(), 0.0);
        std::fill(m->spr_KT.begin(), m->spr_KT.end(), 0.0);
        for (int32_t s = 0; s < ns; ++s) {
            const int32_t i = spr_idx[s];
            if (i < 0 || i >= m->nv || !(spr_k[s] >= 0.0)) return fail(m, PBNG_EINVAL, "bad spring");
            m->spr_K[i] += spr_k[s];
            for (int a = 0; a < 3; ++a) m->spr_KT[3 * (size_t)i + a] += spr_k[s] * spr_target[3 * (size_t)s + a];
        }
        m->has_plane = plane_nd != nullptr && k_contact > 0.0;
        if (m->has_plane) {
            const double n = std::sqrt(plane_nd[0] * plane_nd[0] + plane_nd[1] * plane_nd[1] + plane_nd[2] * plane_nd[2]);
            if (!(n > 0.0)) return fail(m, PBNG_EINVAL, "zero plane normal");
            for (int a = 0; a < 3; ++a) m->pn[a] = plane_nd[a] / n;
            m->pd = plane_nd[3] / n;
            m->kc = k_contact;
        }
        std::fill(m->fext.begin(), m->fext.end(), 0.0);
        if (body_accel)
            for (int32_t e = 0; e < m->ne; ++e) {
                const double rho = density ? density[e] : 1.0;
                for (int j = 0; j < 4; ++j)
                    for (int a = 0; a < 3; ++a)
                        m->fext[3 * (size_t)m->tets[4 * (size_t)e + j] + a] += rho * body_accel[a] * m->vol[e] / 4.0;
            }
    } catch (const std::bad_alloc&) {
        return PBNG_ENOMEM;
    }
    m->dirty = true;
    m->has_state = false;
    return PBNG_OK;
}

pbng_status pbng_set_body_accel(pbng_mesh* m, const double* accel, const double* density) {
    if (!m) return PBNG_EINVAL;
    m->err.clear();
    if (!accel) return fail(m, PBNG_EINVAL, "NULL acceleration");
    std::fill(m->fext.begin(), m->fext.end(), 0.0);
    for (int32_t e = 0; e < m->ne; ++e) {
        const int32_t* t = &m->tets[4 * (size_t)e];
        const int32_t c = m->ncomp > 1 ? m->comp_of[t[0]] : 0;
        const double rho = density ? density[e] : 1.0;
        for (int j = 0; j < 4; ++j)
            for (int a = 0; a < 3; ++a)
                m->fext[3 * (size_t)t[j] + a] += rho * accel[3 * c + a] * m->vol[e] / 4.0;
    }
    m->dirty = true;
    m->has_state = false;
    return PBNG_OK;
}

pbng_status pbng_set_material(pbng_mesh* m, const double* young, const double* poisson) {
    if (!m) return PBNG_EINVAL;
    m->err.clear();
    if (!young || !poisson) return fail(m, PBNG_EINVAL, "NULL material array");
    for (int32_t e = 0; e < m->ne; ++e)
        if (!(young[e] > 0.0) || !(poisson[e] >= 0.0 && poisson[e] < 0.5))
            return fail(m, PBNG_EINVAL, "Young's modulus must be > 0 and 0 <= nu < 0.5");
    for (int32_t e = 0; e < m->ne; ++e) {
        m->mu[e] = young[e] / (2.0 * (1.0 + poisson[e]));                              // Eq. lame
        m->lam[e] = young[e] * poisson[e] / ((1.0 + poisson[e]) * (1.0 - 2.0 * poisson[e]));
    }
    m->dirty = true;
    m->has_state = false;
    return PBNG_OK;
}

pbng_status pbng_set_weak_constraints(pbng_mesh* m, int32_t nc, const int32_t* idx, const double* w,
                                      const double* kn, const double* kt, const double* normal, int32_t recolour) {
    if (!m) return PBNG_EINVAL;
    m->err.clear();
    if (nc < 0 || (nc > 0 && (!idx || !w || !kn || !kt || !normal)))
        return fail(m, PBNG_EINVAL, "bad weak-constraint arrays");
    std::vector<std::vector<int32_t>> cv(nc);
    std::vector<std::vector<double>> cb(nc);
    std::vector<std::array<double, 6>> ck(nc);
    try {
        for (int32_t c = 0; c < nc; ++c) {
            double sum[2] = {0.0, 0.0};
            for (int k = 0; k < 8; ++k) {
                const int32_t v = idx[8 * (size_t)c + k];
                const double wk = w[8 * (size_t)c + k];
                if (v < 0) continue;
                if (v >= m->nv || !(wk >= 0.0)) return fail(m, PBNG_EINVAL, "bad weak-constraint vertex or weight");
                sum[k / 4] += wk;
                const double coef = k < 4 ? wk : -wk;
                size_t q = 0;
                while (q < cv[c].size() && cv[c][q] != v) ++q;
                if (q == cv[c].size()) {
                    cv[c].push_back(v);
                    cb[c].push_back(coef);
                } else {
                    cb[c][q] += coef;
                }
            }
            if (std::fabs(sum[0] - 1.0) > 1e-9 || std::fabs(sum[1] - 1.0) > 1e-9)
                return fail(m, PBNG_EINVAL, "the weights of each side must sum to one");
            if (m->ncomp > 1)
                for (int32_t v : cv[c])
                    if (m->comp_of[v] != m->comp_of[cv[c][0]])
                        return fail(m, PBNG_EINVAL, "a weak constraint joins two components");
            const double* n = normal + 3 * (size_t)c;
            const double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
            if (!(nn > 0.0) || !(kn[c] >= 0.0) || !(kt[c] >= 0.0))
                return fail(m, PBNG_EINVAL, "bad weak-constraint stiffness or normal");
            // K = k_tau I + (k_n - k_tau) n n^T, upper triangle 00 01 02 11 12 22
            const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
            for (int k = 0; k < 6; ++k)
                ck[c][k] = (ia[k] == ib[k] ? kt[c] : 0.0) + (kn[c] - kt[c]) * n[ia[k]] * n[ib[k]] / nn;
        }
    } catch (const std::bad_alloc&) {
        return PBNG_ENOMEM;
    }
    m->wc_v = std::move(cv);
    m->wc_b = std::move(cb);
    m->wc_k = std::move(ck);
    m->wc_incremental = recolour != 0;
    m->dirty = true;
    m->has_state = false;
    return PBNG_OK;
}

pbng_status pbng_set_inertia(pbng_mesh* m, double dt, const double* density) {
    if (!m) return PBNG_EINVAL;
    m->err.clear();
    if (!(dt > 0.0)) {
        if (m->be_dt > 0.0) m->dirty = true;
        m->be_dt = 0.0;
        return PBNG_OK;
    }
    if (!density || !std::isfinite(dt)) return fail(m, PBNG_EINVAL, "backward Euler needs dt > 0 and densities");
    for (int32_t e = 0; e < m->ne; ++e)
        if (!(density[e] > 0.0)) return fail(m, PBNG_EINVAL, "densities must be > 0");
    try {
        m->be_mass.assign(m->nv, 0.0);  // m_ii = sum_e rho_e V_e / 4 (Eq. fem_be, P1)
        for (int32_t e = 0; e < m->ne; ++e)
            for (int j = 0; j < 4; ++j) m->be_mass[m->tets[4 * (size_t)e + j]] += density[e] * m->vol[e] / 4.0;
    } catch (const std::bad_alloc&) {
        return PBNG_ENOMEM;
    }
    m->be_dt = dt;
    m->dirty = true;
    m->has_state = false;
    return PBNG_OK;
}

pbng_status pbng_set_dirichlet_targets(pbng_mesh* m, const double* dir_xyz) {
    if (!m) return PBNG_EINVAL;
    m->err.clear();
    if (!dir_xyz && !m->dir_list.empty()) return fail(m, PBNG_EINVAL, "NULL targets");
    for (size_t q = 0; q < m->dir_list.size(); ++q)
        for (int a = 0; a < 3; ++a) m->dir_pos[3 * (size_t)m->dir_list[q] + a] = dir_xyz[3 * q + a];
    if (m->dirty) return PBNG_OK;  // the next layout build uploads them
    cudaError_t e = cudaSetDevice(m->device);
    if (e != cudaSuccess) return cuda_fail(m, e, "cudaSetDevice");
    const int32_t nd = m->nv - m->nfree;
    std::vector<float4> dhi(nd), dlo(nd);
    for (int32_t q = 0; q < nd; ++q) {
        const int32_t i = m->perm[m->nfree + q];
        float h[3], l[3];
        for (int a = 0; a < 3; ++a) {
            const double d = m->dir_pos[3 * (size_t)i + a] - m->X[3 * (size_t)i + a];
            h[a] = (float)d;
            l[a] = (float)(d - (double)h[a]);
        }
        dhi[q] = make_float4(h[0], h[1], h[2], 0.f);
        dlo[q] = make_float4(l[0], l[1], l[2], 0.f);
    }
    PBNG_CUDA(m, upload(m->d_dir_hi, dhi, m->stream));
    PBNG_CUDA(m, upload(m->d_dir_lo, dlo, m->stream));
    PBNG_CUDA(m, cudaStreamSynchronize(m->stream));
    return PBNG_OK;
}

pbng_status pbng_get_colouring(pbng_mesh* m, int32_t* colour_out, int32_t* ncolours) {
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if (colour_out) std::copy(m->colour.begin(), m->colour.end(), colour_out);
    if (ncolours) *ncolours = m->ncol;
    return PBNG_OK;
}

pbng_status pbng_sweep(pbng_mesh* m, float* u_dev, int32_t nsweeps, const pbng_params* p,
                       double* rel_residual_out) {
    if (!m) return PBNG_EINVAL;
    if (!valid_params(p) || nsweeps < 0) return fail(m, PBNG_EINVAL, "bad parameters");
    if (p->accel == PBNG_ACCEL_CHEBYSHEV && !(p->rho > 0.0))
        return fail(m, PBNG_EINVAL, "automatic rho (rho <= 0) needs the residual checks of pbng_solve");
    select_path(m, p);
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if ((s = check_ext(m, p))) return s;
    if (!u_dev) return fail(m, PBNG_EINVAL, "u_dev is NULL");
    const bool comp = pair_iterate(p->precision);
    if ((s = begin(m, u_dev, p, rel_residual_out != nullptr))) return s;
    // Chunks of up to residual_every sweeps, each one graph launch; the last
    // chunk also computes the residual when it is requested.
    if ((s = ensure_wg(m, (size_t)std::max<int32_t>(1, nsweeps)))) return s;
    const int32_t K = std::min<int32_t>(p->residual_every, kMaxChunk);
    bool res_done = false;
    for (int32_t done = 0; done < nsweeps;) {
        const int32_t chunk = std::min<int32_t>(K, nsweeps - done);
        const bool last = done + chunk == nsweeps;
        // (AUTO reports the extended residual, taken after the chunks)
        const bool with_res = last && rel_residual_out != nullptr && p->precision != PBNG_PREC_AUTO;
        if ((s = run_chunk(m, p, chunk, with_res, m->h_wg + done))) return s;
        res_done = res_done || with_res;
        done += chunk;
    }
    PBNG_CUDA(m, launch_store(m->nv, (const int32_t*)m->d_perm.p, state_of(m, 0), u_dev, m->stream));
    m->kernel_launches++;
    if ((s = check_err(m))) return s;  // synchronises: h_pinned holds the residual
    if (rel_residual_out) {
        std::vector<double> sq(m->ncomp);
        if (res_done) {
            for (int k = 0; k < m->ncomp; ++k) sq[k] = (m->ncol == 0) ? 0.0 : m->h_pinned[k];
        } else if ((s = residual_sq(m, 0, comp, sq.data(), ext_residual(p->precision)))) {
            return s;
        }
        for (int k = 0; k < m->ncomp; ++k)
            rel_residual_out[k] = std::sqrt(sq[k]) / (m->r0[k] > 0 ? m->r0[k] : 1.0);
    }
    return PBNG_OK;
}

pbng_status pbng_sweep_host(pbng_mesh* m, float* u_host, int32_t nsweeps, const pbng_params* p,
                            double* residual_out) {
    if (!m) return PBNG_EINVAL;
    if (!valid_params(p) || nsweeps < 0) return fail(m, PBNG_EINVAL, "bad parameters");
    if (p->accel == PBNG_ACCEL_CHEBYSHEV && !(p->rho > 0.0))
        return fail(m, PBNG_EINVAL, "automatic rho (rho <= 0) needs the residual checks of pbng_solve");
    select_path(m, p);
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if ((s = check_ext(m, p))) return s;
    if (!u_host) return fail(m, PBNG_EINVAL, "u_host is NULL");
    const bool comp = pair_iterate(p->precision);
    const size_t bytes = sizeof(float) * 3 * (size_t)m->nv;
    cudaStream_t st = m->stream;
    PBNG_CUDA(m, ensure_buf(m->d_host_u, bytes));
    float* d_u = (float*)m->d_host_u.p;
    PBNG_CUDA(m, cudaMemcpyAsync(d_u, u_host, bytes, cudaMemcpyHostToDevice, st));
    pbng_params q = *p;
    q.resume = 0;
    m->has_state = false;  // load d_u, fresh acceleration history
    if ((s = begin(m, d_u, &q, false))) return s;
    if ((s = ensure_wg(m, (size_t)std::max<int32_t>(1, nsweeps)))) return s;
    const int32_t K = std::min<int32_t>(q.residual_every, kMaxChunk);
    bool res_done = false;
    for (int32_t done = 0; done < nsweeps;) {
        const int32_t chunk = std::min<int32_t>(K, nsweeps - done);
        const bool with_res = done + chunk == nsweeps && residual_out != nullptr && q.precision != PBNG_PREC_AUTO;
        if ((s = run_chunk(m, &q, chunk, with_res, m->h_wg + done))) return s;
        res_done = res_done || with_res;
        done += chunk;
    }
    if (residual_out && !res_done) {  // no sweep: the residual of the loaded iterate
        const bool multi = m->ncomp > 1;
        if ((s = enqueue_residual(m, state_of(m, 0), comp, (double*)m->d_partial.p, (double*)m->d_comp_sq.p,
                                  (double*)m->d_scalar.p, st, ext_residual(q.precision))))
            return s;
        PBNG_CUDA(m, cudaMemcpyAsync(m->h_pinned, multi ? m->d_comp_sq.p : m->d_scalar.p,
                                     sizeof(double) * (multi ? m->ncomp : 1), cudaMemcpyDeviceToHost, st));
    }
    PBNG_CUDA(m, launch_store(m->nv, (const int32_t*)m->d_perm.p, state_of(m, 0), d_u, st));
    m->kernel_launches++;
    PBNG_CUDA(m, cudaMemcpyAsync(u_host, d_u, bytes, cudaMemcpyDeviceToHost, st));
    if ((s = sync_with_err(m, st))) return s;
    if (residual_out)
        for (int k = 0; k < m->ncomp; ++k) residual_out[k] = (m->ncol == 0) ? 0.0 : std::sqrt(m->h_pinned[k]);
    return PBNG_OK;
}

namespace {

// Automatic Chebyshev rho (pbng_solve, pbng_adjoint): the rho after the
// plain sweeps measured the per-sweep contraction q.
double initial_rho(bool symmetric, double gamma, double q) {
    if (!(q < 1.0)) q = 0.9999;
    if (symmetric) return std::min(kRhoCap, std::max(0.5, 1.0 - gamma * (1.0 - q)));
    return std::min(0.98, std::max(0.5, 1.0 - 2.0 * (1.0 - q)));
}

// The raise rule of the symmetric order: `since` holds (sweeps done, worst
// residual) of the checks since the last (re)start, the last one being the
// current check.  Returns the raised rho, or rho itself.
double raised_rho(const std::vector<std::pair<int32_t, double>>& since, int32_t K, double rho) {
    if (since.size() < 2) return rho;
    const int32_t done = since.back().first;
    const double w = since.back().second;
    const int32_t span = done - since.front().first;
    const int32_t win = std::max<int32_t>(4 * K, (int32_t)std::ceil(3.0 / std::sqrt(2.0 * (1.0 - rho))));
    if (span < win) return rho;
    size_t a = 0;
    while (a + 1 < since.size() && since[a].first - since.front().first < span / 2) ++a;
    const double wa = since[a].second, w0 = since.front().second;
    const int32_t ds = done - since[a].first;
    // still falling over both halves of the window (a floor's fluctuations
    // rarely do), and measurably over the second one
    if (!(ds > 0 && wa > 0.0 && w > 0.0 && w < 0.8 * wa && wa < 0.9 * w0)) return rho;
    const double lam_pred = -std::log(rho / (1.0 + std::sqrt(1.0 - rho * rho)));
    const double lam_obs = -std::log(w / wa) / ds;
    if (!(lam_obs < 0.7 * lam_pred)) return rho;
    const double z = std::exp(lam_pred - lam_obs);
    const double mu = std::min(kRhoCap, rho * 0.5 * (z + 1.0 / z));
    return mu > rho + 0.05 * (1.0 - rho) ? mu : rho;
}

pbng_status solve_impl(pbng_mesh* m, float* u_dev, double rel_tol, int32_t max_sweeps, const pbng_params* p,
                       int32_t* sweeps_out, double* rel_residual_out) {
    if (!valid_params(p) || max_sweeps < 0 || !(rel_tol >= 0.0)) return fail(m, PBNG_EINVAL, "bad parameters");
    select_path(m, p);
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if ((s = check_ext(m, p))) return s;
    if (!u_dev) return fail(m, PBNG_EINVAL, "u_dev is NULL");
    const bool comp = pair_iterate(p->precision);
    if ((s = begin(m, u_dev, p, true))) return s;
    std::vector<double> sq(m->ncomp), rel(m->ncomp, 0.0);
    int32_t done = 0;
    pbng_status result = PBNG_ENOTCONVERGED;
    // With several components each one stops (is frozen: neither updated,
    // accelerated nor re-evaluated) at the first check that finds it below
    // rel_tol, exactly as if it were solved on its own.
    const bool freeze = m->ncomp > 1;
    std::vector<uint8_t> frozen(m->ncomp, 0);
    // Divergence: a non-finite residual, one above kDivergedRel r_0, or one
    // that stays above r_0 after growing kGrowth-fold from the smallest this
    // solve has seen for that component (sustained growth).
    constexpr double kDivergedRel = 1e3, kGrowth = 100.0;
    std::vector<double> least(m->ncomp, 1.0);
    bool changed = false;
    auto converged = [&]() {
        bool all = true;
        changed = false;
        for (int k = 0; k < m->ncomp; ++k) {
            if (frozen[k]) continue;
            rel[k] = std::sqrt(sq[k]) / (m->r0[k] > 0 ? m->r0[k] : 1.0);
            if (!std::isfinite(rel[k]) || rel[k] > kDivergedRel) return -1;
            least[k] = std::min(least[k], rel[k]);
            if (rel[k] > 1.0 && rel[k] > kGrowth * least[k]) return -1;
            if (rel[k] > rel_tol) all = false;
            else if (freeze) {
                frozen[k] = 1;
                m->h_active[k] = 0;
                changed = true;
            }
        }
        return all ? 1 : 0;
    };
    for (int k = 0; k < m->ncomp; ++k) sq[k] = m->r0[k] * m->r0[k];
    int cv = converged();
    if (cv == 1) result = PBNG_OK;
    if (changed && cv == 0)  // components already at rel_tol take no part from the first sweep on
        PBNG_CUDA(m, cudaMemcpyAsync(m->d_active.p, m->h_active, sizeof(int32_t) * m->ncomp,
                                     cudaMemcpyHostToDevice, m->stream));
    const int32_t K = std::min<int32_t>(p->residual_every, kMaxChunk);
    if ((s = ensure_wg(m, (size_t)K))) return s;
    // Chebyshev with rho <= 0: rho from the FP64 residuals.  Plain sweeps
    // first; from the residual ratio over the last two thirds of them, the
    // per-sweep contraction q of the slowest active component.  Ascending
    // colour order: rho = clamp(1 - 2 (1 - q), 0.5, 0.98).  Symmetric order
    // (real spectrum in [0, q]): rho = 1 - gamma (1 - q), the spectral radius
    // of gamma B + (1 - gamma) I, capped at 1 - 1e-6; since the plain rate of
    // a few sweeps underestimates the slowest mode, rho is then raised while
    // the observed Chebyshev rate stays below the one rho predicts (a mode
    // above rho, Manteuffel's adaptive Chebyshev idea): with the predicted
    // per-sweep factor k = rho / (1 + sqrt(1 - rho^2)) and the observed one
    // f > k, that mode sits at rho (z + 1/z) / 2, z = f / k.  Every change
    // restarts the schedule at the current iterate.  A check whose worst
    // residual exceeds 4x the best one seen since the last (re)start backs
    // rho off (1 - rho doubles) and restarts; after kMaxBackoffs the sweeps
    // go plain.
    pbng_params cp = *p;
    const bool auto_rho = p->accel == PBNG_ACCEL_CHEBYSHEV && !(p->rho > 0.0);
    const bool symmetric = p->colour_order == PBNG_ORDER_SYMMETRIC;
    const int32_t est_sweeps = std::max<int32_t>(30, 3 * K);
    constexpr int kMaxBackoffs = 4, kMaxRaises = 12, kMaxEvents = PBNG_MAX_SOLVE_EVENTS;
    int phase = auto_rho ? 0 : 1;
    int32_t mark_done = -1;
    std::vector<double> mark_rel(m->ncomp, 0.0);
    double best = 0.0;
    // checks since the last (re)start: (sweeps done, worst active residual)
    std::vector<std::pair<int32_t, double>> since;
    // PBNG_PREC_AUTO: worst residual of each check while the passes are
    // float32; a window of kStallChecks checks whose best is not below
    // kStallFactor times the best before it, once the residual is below
    // kStallBelow (a slow start is not a floor), is a stall at the float32
    // passes' rounding floor.
    constexpr int kStallChecks = 20;
    constexpr double kStallFactor = 0.5, kStallBelow = 1e-2;
    std::vector<double> stall_hist;
    std::vector<uint8_t> failed_conf(m->ncomp, 0);  // AUTO: a float32 check at tol not confirmed
    auto to_extended = [&]() {
        cp.precision = PBNG_PREC_EXTENDED;
        m->info.extended_from = done;
        stall_hist.clear();
    };
    m->info = pbng_solve_info{};
    m->info.rho = (p->accel == PBNG_ACCEL_CHEBYSHEV && !auto_rho) ? p->rho : 0.0;
    m->info.extended_from = p->precision == PBNG_PREC_EXTENDED ? 0 : -1;
    auto log_event = [&](double rho) {
        if (m->info.nevents < kMaxEvents) {
            m->info.event_sweep[m->info.nevents] = done;
            m->info.event_rho[m->info.nevents] = rho;
            m->info.nevents++;
        }
    };
    if (auto_rho) cp.accel = PBNG_ACCEL_NONE;
    auto restart_history = [&]() -> pbng_status {
        PBNG_CUDA(m, launch_copy_state(m->nv, state_of(m, 0), state_of(m, m->p1_slot), m->stream));
        PBNG_CUDA(m, launch_copy_state(m->nv, state_of(m, 0), state_of(m, m->p2_slot), m->stream));
        m->kernel_launches += 2;
        m->sweep_l = 0;
        m->omega_l = 1.0;
        best = 0.0;
        since.clear();
        log_event(cp.accel == PBNG_ACCEL_CHEBYSHEV ? cp.rho : 0.0);
        return PBNG_OK;
    };
    auto worst_active = [&]() {
        double w = 0.0;
        for (int k = 0; k < m->ncomp; ++k)
            if (!frozen[k]) w = std::max(w, rel[k]);
        return w;
    };
    while (cv == 0 && done < max_sweeps) {
        // one graph launch: the chunk's sweeps and the residual (synchronised
        // below, so the weight staging can be reused)
        int32_t chunk = std::min<int32_t>(K, max_sweeps - done);
        if (phase == 0) chunk = std::min<int32_t>(chunk, est_sweeps - done);
        if ((s = run_chunk(m, &cp, chunk, true, m->h_wg))) return s;
        done += chunk;
        if ((s = check_err(m))) return s;
        for (int k = 0; k < m->ncomp; ++k) sq[k] = (m->ncol == 0) ? 0.0 : m->h_pinned[k];
        if (cp.precision == PBNG_PREC_AUTO) {
            // a float32 check that puts an active component at the tolerance
            // is replaced by the extended residual; the passes go extended
            // once at least half of the active components have failed such a
            // confirmation (they sit at their float32 floor)
            auto below = [&](int k) { return std::sqrt(sq[k]) <= rel_tol * (m->r0[k] > 0 ? m->r0[k] : 1.0); };
            std::vector<uint8_t> was(m->ncomp, 0);
            bool any = false;
            for (int k = 0; k < m->ncomp; ++k)
                if (!frozen[k] && below(k)) was[k] = 1, any = true;
            if (any) {
                if ((s = residual_sq(m, 0, true, sq.data(), true))) return s;
                int failed_active = 0, active = 0;
                for (int k = 0; k < m->ncomp; ++k) {
                    if (was[k] && !below(k)) failed_conf[k] = 1;
                    if (!frozen[k]) {
                        active++;
                        failed_active += failed_conf[k];
                    }
                }
                if (2 * failed_active >= active) to_extended();
            }
        }
        cv = converged();
        if (changed && cv == 0)  // ordered before the next chunk; h_active is not touched until the next sync
            PBNG_CUDA(m, cudaMemcpyAsync(m->d_active.p, m->h_active, sizeof(int32_t) * m->ncomp,
                                         cudaMemcpyHostToDevice, m->stream));
        if (cv == 1) result = PBNG_OK;
        if (cv < 0) result = PBNG_EDIVERGED;
        if (cv != 0) continue;
        const double w = worst_active();
        if (changed) stall_hist.clear();  // the worst active component changed: a new history
        if (cp.precision == PBNG_PREC_AUTO && phase == 1) {
            stall_hist.push_back(w);
            const size_t n = stall_hist.size();
            if (n >= 2 * kStallChecks) {
                const double recent = *std::min_element(stall_hist.end() - kStallChecks, stall_hist.end());
                const double before = *std::min_element(stall_hist.begin(), stall_hist.end() - kStallChecks);
                if (recent > kStallFactor * before && recent < kStallBelow) to_extended();
            }
        }
        if (!auto_rho) continue;
        if (phase == 0) {
            if (mark_done < 0 && 3 * done >= est_sweeps) {
                mark_done = done;
                mark_rel = rel;
            } else if (done >= est_sweeps && mark_done >= 0 && done > mark_done) {
                double q = 0.0;
                for (int k = 0; k < m->ncomp; ++k)
                    if (!frozen[k] && mark_rel[k] > 0.0 && rel[k] > 0.0)
                        q = std::max(q, std::pow(rel[k] / mark_rel[k], 1.0 / (done - mark_done)));
                if (!(q < 1.0)) q = 0.9999;
                cp.accel = PBNG_ACCEL_CHEBYSHEV;
                cp.rho = initial_rho(symmetric, p->gamma, q);
                m->info.plain_rate = q;
                m->info.estimate_sweeps = done;
                m->info.rho = cp.rho;
                phase = 1;
                if ((s = restart_history())) return s;
            }
        } else if (cp.accel == PBNG_ACCEL_CHEBYSHEV) {
            since.emplace_back(done, w);
            if (best == 0.0 || w < best) best = w;
            if (w > 4.0 * best) {
                if (++m->info.restarts > kMaxBackoffs) cp.accel = PBNG_ACCEL_NONE;
                else cp.rho = std::max(0.5, 1.0 - 2.0 * (1.0 - cp.rho));
                m->info.rho = cp.accel == PBNG_ACCEL_CHEBYSHEV ? cp.rho : 0.0;
                if ((s = restart_history())) return s;
            } else if (symmetric && m->info.raises < kMaxRaises) {
                const double mu = raised_rho(since, K, cp.rho);
                if (mu > cp.rho) {
                    cp.rho = mu;
                    m->info.rho = mu;
                    m->info.raises++;
                    if ((s = restart_history())) return s;
                }
            }
        }
    }
    PBNG_CUDA(m, launch_store(m->nv, (const int32_t*)m->d_perm.p, state_of(m, 0), u_dev, m->stream));
    m->kernel_launches++;
    PBNG_CUDA(m, cudaStreamSynchronize(m->stream));
    if (sweeps_out) *sweeps_out = done;
    if (rel_residual_out)
        for (int k = 0; k < m->ncomp; ++k) rel_residual_out[k] = rel[k];
    if (result == PBNG_ENOTCONVERGED) m->err = "max_sweeps reached";
    if (result == PBNG_EDIVERGED) m->err = "residual diverged";
    return result;
}

}  // namespace

pbng_status pbng_solve(pbng_mesh* m, float* u_dev, double rel_tol, int32_t max_sweeps,
                       const pbng_params* p, int32_t* sweeps_out, double* rel_residual_out) {
    if (!m) return PBNG_EINVAL;
    pbng_status r = solve_impl(m, u_dev, rel_tol, max_sweeps, p, sweeps_out, rel_residual_out);
    // A batch's components are frozen one by one as they converge: leave
    // every component active for later calls on every exit path, errors
    // included (after PBNG_ECUDA this is best effort and reports nothing).
    if (m->ncomp > 1 && m->h_active && m->d_active.p) {
        const std::string err = m->err;
        const cudaError_t e1 = cudaStreamSynchronize(m->stream);
        for (int32_t k = 0; k < m->ncomp; ++k) m->h_active[k] = 1;
        const cudaError_t e2 = cudaMemcpyAsync(m->d_active.p, m->h_active, sizeof(int32_t) * m->ncomp,
                                               cudaMemcpyHostToDevice, m->stream);
        const cudaError_t e3 = cudaStreamSynchronize(m->stream);
        if (r == PBNG_OK || r == PBNG_ENOTCONVERGED || r == PBNG_EDIVERGED) {
            if (e1 != cudaSuccess) return cuda_fail(m, e1, "cudaStreamSynchronize");
            if (e2 != cudaSuccess) return cuda_fail(m, e2, "cudaMemcpyAsync");
            if (e3 != cudaSuccess) return cuda_fail(m, e3, "cudaStreamSynchronize");
        }
        m->err = err;
    }
    return r;
}

pbng_status pbng_step(pbng_mesh* m, float* u_dev, float* u_prev_dev, int32_t nsweeps, double rel_tol,
                      const pbng_params* p, int32_t* sweeps_out, double* rel_residual_out) {
    if (!m) return PBNG_EINVAL;
    if (!valid_params(p) || nsweeps < 0 || !(rel_tol >= 0.0)) return fail(m, PBNG_EINVAL, "bad parameters");
    if (!(m->be_dt > 0.0)) return fail(m, PBNG_EINVAL, "pbng_step needs pbng_set_inertia(dt > 0) first");
    if (!u_dev || !u_prev_dev) return fail(m, PBNG_EINVAL, "NULL displacement array");
    select_path(m, p);
    pbng_status s = ensure_ready(m);
    if (s) return s;
    PBNG_CUDA(m, launch_inertia(m->nv, m->nfree, (const int32_t*)m->d_perm.p, u_dev, u_prev_dev,
                                (const float4*)m->d_aux_base0.p, (const float4*)m->d_aux_base1.p,
                                (const float*)m->d_be_k.p, (float4*)m->d_aux0.p, (float4*)m->d_aux1.p, m->stream));
    m->kernel_launches++;
    pbng_params q = *p;
    q.resume = 0;
    if (rel_tol > 0.0) return pbng_solve(m, u_dev, rel_tol, nsweeps, &q, sweeps_out, rel_residual_out);
    s = pbng_sweep(m, u_dev, nsweeps, &q, rel_residual_out);
    if (s == PBNG_OK && sweeps_out) *sweeps_out = nsweeps;
    return s;
}

}  // extern "C"

namespace {

// Per-tet data and buffers of the adjoint (once per layout).
pbng_status adjoint_setup(pbng_mesh* m) {
    if (m->adj_ready) return PBNG_OK;
    cudaStream_t st = m->stream;
    std::vector<int32_t> iperm(m->nv);
    for (int32_t w = 0; w < m->nv; ++w) iperm[m->perm[w]] = w;
    std::vector<int4> tv(m->ne);
    std::vector<float4> tb(3 * (size_t)m->ne);
    for (int32_t e = 0; e < m->ne; ++e) {
        const int32_t* t = &m->tets[4 * (size_t)e];
        tv[e] = make_int4(iperm[t[0]], iperm[t[1]], iperm[t[2]], iperm[t[3]]);
        const double* B = &m->B[9 * (size_t)e];
        tb[3 * (size_t)e] = make_float4((float)B[0], (float)B[1], (float)B[2], (float)(2.0 * m->mu[e] * m->vol[e]));
        tb[3 * (size_t)e + 1] = make_float4((float)B[3], (float)B[4], (float)B[5], (float)(m->lam[e] * m->vol[e]));
        tb[3 * (size_t)e + 2] = make_float4((float)B[6], (float)B[7], (float)B[8], 0.f);
    }
    const int32_t nd = (int32_t)m->dir_list.size();
    std::vector<int32_t> dq_int(nd), dq_caller(m->dir_list);
    for (int32_t q = 0; q < nd; ++q) dq_int[q] = iperm[m->dir_list[q]];
    PBNG_CUDA(m, upload(m->d_tv, tv, st));
    PBNG_CUDA(m, upload(m->d_tb, tb, st));
    PBNG_CUDA(m, upload(m->d_dq_int, dq_int, st));
    PBNG_CUDA(m, upload(m->d_dq_caller, dq_caller, st));
    for (auto& b : m->d_lam) PBNG_CUDA(m, ensure_buf(b, sizeof(float4) * (size_t)m->nv));
    PBNG_CUDA(m, ensure_buf(m->d_gv, sizeof(float4) * (size_t)std::max(1, m->nfree)));
    PBNG_CUDA(m, ensure_buf(m->d_diag, 2 * sizeof(float4) * (size_t)std::max(1, m->nfree)));
    PBNG_CUDA(m, ensure_buf(m->d_hdl, sizeof(float4) * (size_t)m->nv));
    // per-warp partials of the direct-load kernels and of the pipelined
    // Hessian action, whose grids differ
    PBNG_CUDA(m, ensure_buf(m->d_adj_partial,
                            sizeof(double) * (size_t)std::max({1, adjoint_warps(m->nitems_ring),
                                                               adjoint_ring_apply_warps(m->nitems_ring)})));
    double vmin = 0.0;
    for (int32_t e = 0; e < m->ne; ++e) vmin = (e == 0) ? m->vol[e] : std::min(vmin, m->vol[e]);
    m->h_min = std::cbrt(6.0 * vmin);
    m->adj_ready = true;
    return PBNG_OK;
}

// FP64 |rhs - H lambda|^2 -> host.
pbng_status adjoint_resid(pbng_mesh* m, State u, float4* lam, const float4* rhs, double* out) {
    cudaStream_t st = m->stream;
    PBNG_CUDA(m, launch_adjoint_vertex(kAdjResid, m->dm, u, lam, rhs, (float4*)m->d_diag.p,
                                       (const Item*)m->d_items.p, m->nitems_ring, (int32_t*)m->d_err.p,
                                       (double*)m->d_adj_partial.p, st, nullptr, m->model));
    PBNG_CUDA(m, launch_reduce((const double*)m->d_adj_partial.p, adjoint_warps(m->nitems_ring),
                               (double*)m->d_scalar.p, st));
    m->kernel_launches += 2;
    PBNG_CUDA(m, cudaMemcpyAsync(m->h_pinned, m->d_scalar.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    PBNG_CUDA(m, cudaStreamSynchronize(st));
    *out = m->h_pinned[0];
    return PBNG_OK;
}

}  // namespace

namespace {

// Buffers of the Newton-CG solver and of pbng_force / pbng_hessian_apply.
pbng_status newton_setup(pbng_mesh* m) {
    pbng_status s = adjoint_setup(m);
    if (s) return s;
    for (auto& b : m->d_nw) PBNG_CUDA(m, ensure_buf(b, sizeof(float4) * (size_t)m->nv));
    const size_t np = (size_t)std::max({1, vec_blocks(m->nfree), adjoint_warps(m->nitems_ring),
                                        adjoint_ring_apply_warps(m->nitems_ring)});
    for (auto& b : m->d_nw_part) PBNG_CUDA(m, ensure_buf(b, sizeof(double) * np));
    PBNG_CUDA(m, ensure_buf(m->d_nw_sc, sizeof(double) * 4));
    PBNG_CUDA(m, ensure_buf(m->d_nw_flag, sizeof(int32_t)));
    if (!m->h_nw) PBNG_CUDA(m, cudaMallocHost((void**)&m->h_nw, sizeof(double) * 2));
    return PBNG_OK;
}

// Checks shared by the Newton-CG entry points: corotated, ring layout.
pbng_status newton_ready(pbng_mesh* m, const pbng_params* p) {
    if (!valid_params(p)) return fail(m, PBNG_EINVAL, "bad parameters");
    if (p->kernel_path != 0) return fail(m, PBNG_EINVAL, "Newton-CG runs on the ring layout (kernel_path 0)");
    select_path(m, p);
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if (!m->all_ring) return fail(m, PBNG_EINVAL, "Newton-CG needs every colour in the ring layout");
    return newton_setup(m);
}

// r = f + f^ext at state u into d_nw[0], the SPD blocks into d_diag; FP64 |r|^2 -> *rr.
pbng_status newton_force(pbng_mesh* m, State u, double* rr) {
    cudaStream_t st = m->stream;
    float4* r = (float4*)m->d_nw[0].p;
    PBNG_CUDA(m, launch_adjoint_vertex(kAdjForce, m->dm, u, nullptr, nullptr, (float4*)m->d_diag.p,
                                       (const Item*)m->d_items.p, m->nitems_ring, (int32_t*)m->d_err.p,
                                       (double*)m->d_nw_part[0].p, st, r, m->model));
    PBNG_CUDA(m, launch_reduce((const double*)m->d_nw_part[0].p, adjoint_warps(m->nitems_ring),
                               (double*)m->d_scalar.p, st));
    m->kernel_launches += 2;
    PBNG_CUDA(m, cudaMemcpyAsync(m->h_pinned, m->d_scalar.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    PBNG_CUDA(m, cudaStreamSynchronize(st));
    *rr = m->h_pinned[0];
    return check_err(m);
}

}  // namespace

extern "C" {

pbng_status pbng_adjoint(pbng_mesh* m, const float* u_eq_dev, const float* dLdu_dev, float* dL_dlogE_dev,
                         float* dL_dxD_dev, double rel_tol, int32_t max_sweeps, const pbng_params* p,
                         int32_t* sweeps_out, double* rel_residual_out) {
    if (!m) return PBNG_EINVAL;
    // PBNG_ACCEL_CG (this entry point only): conjugate gradients with one
    // symmetric block Gauss-Seidel sweep as the preconditioner
    const bool cg = p && p->accel == PBNG_ACCEL_CG;
    pbng_params pv{};
    if (p) {
        pv = *p;
        if (cg) pv.accel = PBNG_ACCEL_NONE;
    }
    if (!p || !valid_params(&pv) || max_sweeps < 0 || !(rel_tol >= 0.0)) return fail(m, PBNG_EINVAL, "bad parameters");
    if (cg && p->colour_order != PBNG_ORDER_SYMMETRIC)
        return fail(m, PBNG_EINVAL, "conjugate gradients need the symmetric colour order (a symmetric preconditioner)");
    if (!u_eq_dev || !dLdu_dev || !dL_dlogE_dev) return fail(m, PBNG_EINVAL, "NULL argument");
    if (p->kernel_path != 0) return fail(m, PBNG_EINVAL, "the adjoint runs on the ring layout (kernel_path 0)");
    select_path(m, p);
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if (!m->all_ring) return fail(m, PBNG_EINVAL, "the adjoint needs every colour in the ring layout");
    if ((s = adjoint_setup(m))) return s;
    cudaStream_t st = m->stream;
    const bool refine = p->precision == PBNG_PREC_EXTENDED || p->precision == PBNG_PREC_AUTO;
    // u_eq -> state slot 3 (clamped vertices at their targets)
    PBNG_CUDA(m, launch_load(m->nv, m->nfree, u_eq_dev, (const int32_t*)m->d_perm.p, (const float4*)m->d_dir_hi.p,
                             (const float4*)m->d_dir_lo.p, state_of(m, 3), st));
    PBNG_CUDA(m, launch_gather_rhs(m->nfree, (const int32_t*)m->d_perm.p, dLdu_dev, (float4*)m->d_gv.p, st));
    for (auto& b : m->d_lam) PBNG_CUDA(m, cudaMemsetAsync(b.p, 0, sizeof(float4) * (size_t)m->nv, st));
    const State u = state_of(m, 3);
    float4* lam = (float4*)m->d_lam[0].p;
    PBNG_CUDA(m, launch_adjoint_vertex(kAdjDiag, m->dm, u, lam, (const float4*)m->d_gv.p, (float4*)m->d_diag.p,
                                       (const Item*)m->d_items.p, m->nitems_ring, (int32_t*)m->d_err.p, nullptr, st,
                                       nullptr, m->model));
    m->kernel_launches += 3;
    double g2 = 0.0;
    if ((s = adjoint_resid(m, u, lam, (const float4*)m->d_gv.p, &g2))) return s;  // lambda = 0: |dL/du|^2
    // Gauss-Seidel sweeps with the forward's acceleration, on a local sweep
    // index so the forward iterate's history is left alone
    const int32_t saved_l = m->sweep_l;
    const double saved_om = m->omega_l;
    int32_t done = 0;
    double rel = g2 > 0.0 ? 1.0 : 0.0;
    pbng_status result = PBNG_ENOTCONVERGED;
    const int32_t K = std::min<int32_t>(p->residual_every, kMaxChunk);
    if ((s = ensure_wg(m, (size_t)K))) return s;
    const std::vector<int> seq = colour_sequence(m->ncol, p->colour_order);
    // Automatic rho (Chebyshev with rho <= 0) as in pbng_solve: plain sweeps
    // measure q, then Chebyshev from rho(q), raised (symmetric order) or
    // backed off (growth) with a restart of the multiplier history.  The
    // estimate carries over from one inner solve to the next (same H).
    pbng_params cp = *p;
    const bool auto_rho = p->accel == PBNG_ACCEL_CHEBYSHEV && !(p->rho > 0.0);
    const bool symmetric = p->colour_order == PBNG_ORDER_SYMMETRIC;
    const int32_t est_sweeps = std::max<int32_t>(30, 3 * K);
    int phase = auto_rho ? 0 : 1, backoffs = 0, raises = 0;
    if (auto_rho) cp.accel = PBNG_ACCEL_NONE;
    // One block Gauss-Seidel solve of H lam = rhs from lam = 0, until its
    // float32 relative residual is <= tol, or (stall) its best over the last
    // kStall checks is not below half the best before them, or the budget.
    constexpr int kStall = 10;
    auto inner_solve = [&](const float4* rhs, double rhs2, double tol, bool stall_stop, double* rel_end) -> pbng_status {
        for (auto& b : m->d_lam) PBNG_CUDA(m, cudaMemsetAsync(b.p, 0, sizeof(float4) * (size_t)m->nv, st));
        m->sweep_l = 0;
        m->omega_l = 1.0;
        int p1 = 1, p2 = 2;
        int32_t mark_done = -1, start = done;
        double mark_rel = 0.0, best = 0.0, r2 = 0.0, irel = 1.0;
        std::vector<std::pair<int32_t, double>> since;
        std::vector<double> hist;
        auto restart = [&]() -> pbng_status {
            for (int q = 1; q <= 2; ++q)
                PBNG_CUDA(m, cudaMemcpyAsync(m->d_lam[q].p, lam, sizeof(float4) * (size_t)m->nv,
                                             cudaMemcpyDeviceToDevice, st));
            m->sweep_l = 0;
            m->omega_l = 1.0;
            best = 0.0;
            since.clear();
            return PBNG_OK;
        };
        while (rhs2 > 0.0 && done < max_sweeps) {
            int32_t chunk = std::min<int32_t>(K, max_sweeps - done);
            if (phase == 0) chunk = std::min<int32_t>(chunk, start + est_sweeps - done);
            chunk_weights(m, &cp, chunk, m->h_wg);
            PBNG_CUDA(m, cudaMemcpyAsync(m->d_wg.p, m->h_wg, sizeof(float2) * chunk, cudaMemcpyHostToDevice, st));
            for (int32_t k = 0; k < chunk; ++k) {
                for (const int c : seq)
                    PBNG_CUDA(m, launch_adjoint_ring_sweep(m->dm, u, lam, rhs, (const float4*)m->d_diag.p,
                                                           (const Item*)m->d_items.p + m->item_off[c],
                                                           m->item_off[c + 1] - m->item_off[c], (int32_t*)m->d_err.p,
                                                           m->model, st));
                m->kernel_launches += (int64_t)seq.size();
                if (cp.accel != PBNG_ACCEL_NONE && m->nfree > 0) {
                    const State lc{lam, lam}, l1{(float4*)m->d_lam[p1].p, (float4*)m->d_lam[p1].p},
                        l2{(float4*)m->d_lam[p2].p, (float4*)m->d_lam[p2].p};
                    PBNG_CUDA(m, launch_accel(m->nfree, lc, l1, l2, (const float2*)m->d_wg.p + k, nullptr, nullptr,
                                              false, st));
                    m->kernel_launches++;
                    std::swap(p1, p2);
                }
            }
            done += chunk;
            pbng_status e = check_err(m);
            if (e) return e;
            if ((e = adjoint_resid(m, u, lam, rhs, &r2))) return e;
            irel = std::sqrt(r2 / rhs2);
            *rel_end = irel;
            if (!std::isfinite(irel) || irel > 1e3) return PBNG_EDIVERGED;
            if (irel <= tol) return PBNG_OK;
            hist.push_back(irel);
            if (stall_stop && hist.size() >= 2 * kStall) {
                const double recent = *std::min_element(hist.end() - kStall, hist.end());
                const double before = *std::min_element(hist.begin(), hist.end() - kStall);
                if (recent > 0.5 * before) return PBNG_OK;  // at this solve's float32 floor
            }
            if (!auto_rho) continue;
            if (phase == 0) {
                if (mark_done < 0 && 3 * (done - start) >= est_sweeps) {
                    mark_done = done;
                    mark_rel = irel;
                } else if (done - start >= est_sweeps && mark_done >= 0 && done > mark_done) {
                    const double q = mark_rel > 0.0 && irel > 0.0 ? std::pow(irel / mark_rel, 1.0 / (done - mark_done))
                                                                  : 0.0;
                    cp.accel = PBNG_ACCEL_CHEBYSHEV;
                    cp.rho = initial_rho(symmetric, p->gamma, q);
                    phase = 1;
                    if ((e = restart())) return e;
                }
            } else if (cp.accel == PBNG_ACCEL_CHEBYSHEV) {
                since.emplace_back(done, irel);
                if (best == 0.0 || irel < best) best = irel;
                if (irel > 4.0 * best) {
                    if (++backoffs > 4) cp.accel = PBNG_ACCEL_NONE;
                    else cp.rho = std::max(0.5, 1.0 - 2.0 * (1.0 - cp.rho));
                    if ((e = restart())) return e;
                } else if (symmetric && raises < 12) {
                    const double mu = raised_rho(since, K, cp.rho);
                    if (mu > cp.rho) {
                        cp.rho = mu;
                        raises++;
                        if ((e = restart())) return e;
                    }
                }
            }
        }
        return rhs2 > 0.0 ? PBNG_ENOTCONVERGED : PBNG_OK;
    };
    // Conjugate gradients on H d = rhs from d = 0 (in lam), preconditioned by
    // one symmetric block Gauss-Seidel sweep from zero (the sweeps above
    // with rhs in place of dL/du: z = M^{-1} r with M = (D + L) D^{-1}
    // (D + L^T), symmetric positive definite with H).  Each iteration is one
    // preconditioner sweep and one Hessian action, counted as one sweep;
    // the recursive residual r decides the stop (tol of rhs, a stall, or
    // the budget).  FP64 dot products kept on the device, float32 vectors.
    if (cg) {
        const size_t fb = sizeof(float4) * (size_t)std::max(1, m->nfree);
        for (auto& b : m->d_acg) PBNG_CUDA(m, ensure_buf(b, fb));
        for (auto& b : m->d_acg_part)
            PBNG_CUDA(m, ensure_buf(b, sizeof(double) * (size_t)std::max(1, adj_vec_blocks(m->nfree))));
        PBNG_CUDA(m, ensure_buf(m->d_acg_sc, 5 * sizeof(double)));
    }
    auto inner_cg = [&](const float4* rhs, double rhs2, double tol, bool stall_stop, double* rel_end) -> pbng_status {
        float4* x = lam;
        float4* pdir = (float4*)m->d_lam[1].p;
        float4* z = (float4*)m->d_lam[2].p;
        float4* r = (float4*)m->d_acg[0].p;
        float4* q = (float4*)m->d_acg[1].p;
        double* sc = (double*)m->d_acg_sc.p;  // r.z, p.Hp, new r.z, |r|^2
        int32_t* flag = (int32_t*)(sc + 4);
        const int nb = adj_vec_blocks(m->nfree), na = adjoint_ring_apply_warps(m->nitems_ring);
        const size_t vb = sizeof(float4) * (size_t)m->nv, fb = sizeof(float4) * (size_t)m->nfree;
        for (float4* b : {x, pdir}) PBNG_CUDA(m, cudaMemsetAsync(b, 0, vb, st));
        PBNG_CUDA(m, cudaMemsetAsync(sc, 0, 5 * sizeof(double), st));
        PBNG_CUDA(m, cudaMemcpyAsync(r, rhs, fb, cudaMemcpyDeviceToDevice, st));
        auto precondition = [&](double* rz_out) -> pbng_status {  // z = M^{-1} r, r . z -> *rz_out
            PBNG_CUDA(m, cudaMemsetAsync(z, 0, vb, st));
            for (const int c : seq)
                PBNG_CUDA(m, launch_adjoint_ring_sweep(m->dm, u, z, r, (const float4*)m->d_diag.p,
                                                       (const Item*)m->d_items.p + m->item_off[c],
                                                       m->item_off[c + 1] - m->item_off[c], (int32_t*)m->d_err.p,
                                                       m->model, st));
            PBNG_CUDA(m, launch_acg_dot(m->nfree, r, z, (double*)m->d_acg_part[1].p, st));
            PBNG_CUDA(m, launch_reduce((const double*)m->d_acg_part[1].p, nb, rz_out, st));
            m->kernel_launches += (int64_t)seq.size() + 2;
            return PBNG_OK;
        };
        pbng_status e;
        if ((e = precondition(sc))) return e;
        PBNG_CUDA(m, cudaMemcpyAsync(pdir, z, fb, cudaMemcpyDeviceToDevice, st));
        // The scalars stay on the device; the host reads |r|^2 and the
        // breakdown flag every kCheck iterations (and at the budget's end).
        constexpr int kCheck = 8;
        constexpr size_t kStallChecks = 7;  // a stall over about 56 iterations
        std::vector<double> hist;
        int it = 0;
        while (rhs2 > 0.0 && done < max_sweeps) {
            // q = H p and p . H p (the pipelined action over every ring item)
            PBNG_CUDA(m, launch_adjoint_ring_apply(m->dm, u, pdir, (const Item*)m->d_items.p, m->nitems_ring,
                                                   (int32_t*)m->d_err.p, m->model, q, (double*)m->d_adj_partial.p,
                                                   st));
            PBNG_CUDA(m, launch_reduce((const double*)m->d_adj_partial.p, na, sc + 1, st));
            PBNG_CUDA(m, launch_acg_step(m->nfree, sc, flag, pdir, q, x, r, (double*)m->d_acg_part[0].p, st));
            PBNG_CUDA(m, launch_reduce((const double*)m->d_acg_part[0].p, nb, sc + 3, st));
            m->kernel_launches += 4;
            if ((e = precondition(sc + 2))) return e;
            PBNG_CUDA(m, launch_cg_dir(m->nfree, sc, z, pdir, flag, sc, st));  // p = z + b p; sc[0] = sc[2]
            m->kernel_launches += 2;
            done++;
            if (++it % kCheck != 0 && done < max_sweeps) continue;
            PBNG_CUDA(m, cudaMemcpyAsync(m->h_pinned, sc + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
            if ((e = sync_with_err(m, st))) return e;
            int32_t f = 0;
            std::memcpy(&f, m->h_pinned + 1, sizeof(int32_t));
            // a non-positive curvature: H is not positive definite here
            if (f) return PBNG_EDIVERGED;
            const double irel = std::sqrt(m->h_pinned[0] / rhs2);
            *rel_end = irel;
            if (!std::isfinite(irel) || irel > 1e3) return PBNG_EDIVERGED;
            if (irel <= tol) return PBNG_OK;
            // a stall: the best of the last kStallChecks checks not below half
            // the best before them
            hist.push_back(irel);
            if (stall_stop && hist.size() >= 2 * kStallChecks) {
                const double recent = *std::min_element(hist.end() - kStallChecks, hist.end());
                const double before = *std::min_element(hist.begin(), hist.end() - kStallChecks);
                if (recent > 0.5 * before) return PBNG_OK;
            }
        }
        return rhs2 > 0.0 ? PBNG_ENOTCONVERGED : PBNG_OK;
    };
    if (cg && !refine) {
        // one float32 solve; the reported residual is the true one
        double irel = rel;
        s = inner_cg((const float4*)m->d_gv.p, g2, rel_tol, false, &irel);
        if (s == PBNG_OK || s == PBNG_ENOTCONVERGED || s == PBNG_EDIVERGED) {
            result = s;
            s = PBNG_OK;
            double r2 = 0.0;
            if (g2 > 0.0 && result != PBNG_EDIVERGED && !(s = adjoint_resid(m, u, lam, (const float4*)m->d_gv.p, &r2))) {
                rel = std::sqrt(r2 / g2);
                if (result == PBNG_OK && rel > rel_tol) result = PBNG_ENOTCONVERGED;
            }
        }
    } else if (!refine) {
        double irel = rel;
        s = inner_solve((const float4*)m->d_gv.p, g2, rel_tol, false, &irel);
        if (g2 > 0.0) rel = irel;
        if (s == PBNG_OK || s == PBNG_ENOTCONVERGED || s == PBNG_EDIVERGED) {
            result = s;
            s = PBNG_OK;
        }
    } else {
        // Mixed-precision iterative refinement (the adjoint is linear): the
        // multipliers accumulate as float pairs, the residual dL/du - H lam
        // is formed by central differences of the float-float force,
        // H lam = -(F(u + eps lam) - F(u - eps lam)) / (2 eps), and each
        // correction solves H d = residual with the float32 sweeps to 1e-2
        // or to their floor.  eps makes the largest step eps |lam| 1e-4 of
        // the smallest element size, where the central difference's error
        // (~(eps |lam| / h)^2) is below the forces' rounding.
        const size_t vbytes = sizeof(float4) * (size_t)m->nv;
        PBNG_CUDA(m, ensure_buf(m->d_lam_hi, vbytes));
        PBNG_CUDA(m, ensure_buf(m->d_lam_lo, vbytes));
        PBNG_CUDA(m, ensure_buf(m->d_rhs, sizeof(float4) * (size_t)std::max(1, m->nfree)));
        for (auto* b : {&m->d_fp[0], &m->d_fp[1], &m->d_fp[2], &m->d_fp[3]})
            PBNG_CUDA(m, ensure_buf(*b, sizeof(float4) * (size_t)std::max(1, m->nfree)));
        for (auto& sb : m->d_shift)
            for (auto& b : sb) PBNG_CUDA(m, ensure_buf(b, vbytes));
        PBNG_CUDA(m, ensure_buf(m->d_maxabs, sizeof(float) * 4));
        PBNG_CUDA(m, ensure_buf(m->d_refine_partial, sizeof(double) * (size_t)std::max(1, adj_vec_blocks(m->nfree))));
        PBNG_CUDA(m, cudaMemsetAsync(m->d_lam_hi.p, 0, vbytes, st));
        PBNG_CUDA(m, cudaMemsetAsync(m->d_lam_lo.p, 0, vbytes, st));
        PBNG_CUDA(m, cudaMemcpyAsync(m->d_rhs.p, m->d_gv.p, sizeof(float4) * (size_t)m->nfree, cudaMemcpyDeviceToDevice,
                                     st));
        const State up{(float4*)m->d_shift[0][0].p, (float4*)m->d_shift[0][1].p};
        const State um{(float4*)m->d_shift[1][0].p, (float4*)m->d_shift[1][1].p};
        double r2 = g2;
        result = g2 > 0.0 ? PBNG_ENOTCONVERGED : PBNG_OK;
        while (g2 > 0.0 && done < max_sweeps && s == PBNG_OK) {
            double irel = 1.0;
            // each correction to 1e-2 (sweeps) or 1e-3 (conjugate gradients) of
            // its right-hand side, both above the float32 floor of H d, or only
            // to half of what is left to rel_tol when that is less
            const double left = 0.5 * rel_tol * std::sqrt(g2 / r2);
            pbng_status is = cg ? inner_cg((const float4*)m->d_rhs.p, r2, std::max(1e-3, left), true, &irel)
                                : inner_solve((const float4*)m->d_rhs.p, r2, std::max(1e-2, left), true, &irel);
            if (is == PBNG_EDIVERGED) { result = is; break; }
            if (is != PBNG_OK && is != PBNG_ENOTCONVERGED) { s = is; break; }
            // lam += d, then the residual at the new lam
            PBNG_CUDA(m, cudaMemsetAsync(m->d_maxabs.p, 0, sizeof(float), st));
            PBNG_CUDA(m, launch_adjoint_accumulate(m->nfree, lam, (float4*)m->d_lam_hi.p, (float4*)m->d_lam_lo.p,
                                                   (float*)m->d_maxabs.p, st));
            float maxabs = 0.0f;
            PBNG_CUDA(m, cudaMemcpyAsync(&maxabs, m->d_maxabs.p, sizeof(float), cudaMemcpyDeviceToHost, st));
            PBNG_CUDA(m, cudaStreamSynchronize(st));
            if (!(maxabs > 0.0f) || !std::isfinite(maxabs)) { result = PBNG_EDIVERGED; break; }
            const float eps = (float)(1e-4 * m->h_min / (double)maxabs);
            PBNG_CUDA(m, launch_adjoint_shift(m->nv, u, (const float4*)m->d_lam_hi.p, (const float4*)m->d_lam_lo.p, eps,
                                              up, um, st));
            for (int k = 0; k < 2; ++k) {
                DeviceMesh d = m->dm;
                d.fout_hi = (float4*)m->d_fp[2 * k].p;
                d.fout_lo = (float4*)m->d_fp[2 * k + 1].p;
                d.vsq = nullptr;
                PBNG_CUDA(m, launch_ring_residual(d, k == 0 ? up : um, (const Item*)m->d_items.p, m->nitems_ring, true,
                                                  (double*)m->d_partial.p, nullptr, m->model, (int32_t*)m->d_err.p, st,
                                                  true, m->ring_partials));
            }
            PBNG_CUDA(m, launch_adjoint_refine_rhs(m->nfree, (const float4*)m->d_gv.p, (const float4*)m->d_fp[0].p,
                                                   (const float4*)m->d_fp[1].p, (const float4*)m->d_fp[2].p,
                                                   (const float4*)m->d_fp[3].p, 0.5 / (double)eps, (float4*)m->d_rhs.p,
                                                   (double*)m->d_refine_partial.p, st));
            PBNG_CUDA(m, launch_reduce((const double*)m->d_refine_partial.p, adj_vec_blocks(m->nfree),
                                       (double*)m->d_scalar.p, st));
            m->kernel_launches += 6;
            PBNG_CUDA(m, cudaMemcpyAsync(m->h_pinned, m->d_scalar.p, sizeof(double), cudaMemcpyDeviceToHost, st));
            if ((s = sync_with_err(m, st))) break;
            r2 = m->h_pinned[0];
            rel = std::sqrt(r2 / g2);
            if (!std::isfinite(rel) || rel > 1e3) { result = PBNG_EDIVERGED; break; }
            if (rel <= rel_tol) { result = PBNG_OK; break; }
        }
        lam = (float4*)m->d_lam_hi.p;  // the gradients use the accumulated multipliers
    }
    m->sweep_l = saved_l;
    m->omega_l = saved_om;
    if (s) return s;
    if (g2 == 0.0) result = PBNG_OK;
    // sensitivities
    PBNG_CUDA(m, cudaMemsetAsync(m->d_hdl.p, 0, sizeof(float4) * (size_t)m->nv, st));
    PBNG_CUDA(m, launch_adjoint_tets(m->ne, m->nfree, (const int4*)m->d_tv.p, (const float4*)m->d_tb.p, u, lam,
                                     dL_dlogE_dev, (float*)m->d_hdl.p, st, m->model));
    PBNG_CUDA(m, launch_adjoint_weak_clamped((int)m->wc_v.size(), m->nfree, m->dm, lam, (float*)m->d_hdl.p, st));
    m->kernel_launches += m->wc_v.empty() ? 1 : 2;
    if (dL_dxD_dev) {
        PBNG_CUDA(m, launch_clamped_grad((int32_t)m->dir_list.size(), (const int32_t*)m->d_dq_int.p,
                                         (const int32_t*)m->d_dq_caller.p, dLdu_dev, (const float*)m->d_hdl.p,
                                         dL_dxD_dev, st));
        m->kernel_launches++;
    }
    if ((s = check_err(m))) return s;
    if (sweeps_out) *sweeps_out = done;
    if (rel_residual_out) *rel_residual_out = rel;
    if (result == PBNG_ENOTCONVERGED) m->err = "max_sweeps reached";
    if (result == PBNG_EDIVERGED) m->err = "adjoint iteration diverged";
    return result;
}

pbng_status pbng_force(pbng_mesh* m, const float* u_dev, const pbng_params* p, float* f_out_dev) {
    if (!m) return PBNG_EINVAL;
    pbng_params dp;
    if (!p) {
        pbng_default_params(&dp);
        p = &dp;
    }
    if (!u_dev || !f_out_dev) return fail(m, PBNG_EINVAL, "NULL argument");
    pbng_status s = newton_ready(m, p);
    if (s) return s;
    cudaStream_t st = m->stream;
    PBNG_CUDA(m, launch_load(m->nv, m->nfree, u_dev, (const int32_t*)m->d_perm.p, (const float4*)m->d_dir_hi.p,
                             (const float4*)m->d_dir_lo.p, state_of(m, 3), st));
    double rr = 0.0;
    if ((s = newton_force(m, state_of(m, 3), &rr))) return s;
    PBNG_CUDA(m, launch_scatter_vec(m->nv, m->nfree, (const int32_t*)m->d_perm.p, (const float4*)m->d_nw[0].p,
                                    f_out_dev, st));
    m->kernel_launches += 2;
    return check_err(m);  // synchronises
}

pbng_status pbng_hessian_apply(pbng_mesh* m, const float* u_dev, const float* p_dev, const pbng_params* p,
                               float* hp_out_dev) {
    if (!m) return PBNG_EINVAL;
    pbng_params dp;
    if (!p) {
        pbng_default_params(&dp);
        p = &dp;
    }
    if (!u_dev || !p_dev || !hp_out_dev) return fail(m, PBNG_EINVAL, "NULL argument");
    pbng_status s = newton_ready(m, p);
    if (s) return s;
    cudaStream_t st = m->stream;
    const int32_t* perm = (const int32_t*)m->d_perm.p;
    PBNG_CUDA(m, launch_load(m->nv, m->nfree, u_dev, perm, (const float4*)m->d_dir_hi.p,
                             (const float4*)m->d_dir_lo.p, state_of(m, 3), st));
    PBNG_CUDA(m, launch_gather_vec(m->nv, m->nfree, perm, p_dev, (float4*)m->d_nw[3].p, st));
    PBNG_CUDA(m, launch_adjoint_ring_apply(m->dm, state_of(m, 3), (float4*)m->d_nw[3].p, (const Item*)m->d_items.p,
                                           m->nitems_ring, (int32_t*)m->d_err.p, m->model, (float4*)m->d_nw[4].p,
                                           (double*)m->d_nw_part[0].p, st));
    PBNG_CUDA(m, launch_scatter_vec(m->nv, m->nfree, perm, (const float4*)m->d_nw[4].p, hp_out_dev, st));
    m->kernel_launches += 4;
    PBNG_CUDA(m, cudaStreamSynchronize(st));
    return check_err(m);
}

// Newton's method on f(u) + f^ext = 0 with the true Hessian (Eq. hess) and a
// block-Jacobi preconditioned CG inner solve, truncated at the first
// direction of non-positive curvature; a backtracking line search halves the
// step until |r| decreases by the factor (1 - 1e-4 s).  If no step along the
// CG direction is accepted, the preconditioned residual D^{-1} r (the
// Jacobi counterpart of one PBNG sweep) is tried instead.
pbng_status pbng_newton_cg(pbng_mesh* m, float* u_dev, double rel_tol, int32_t max_newton, int32_t max_cg,
                           double cg_tol, const pbng_params* p, pbng_newton_info* info) {
    if (!m) return PBNG_EINVAL;
    if (!p || !u_dev || !(rel_tol >= 0.0) || max_newton < 0 || max_cg < 1 || !(cg_tol > 0.0 && cg_tol < 1.0))
        return fail(m, PBNG_EINVAL, "bad Newton-CG arguments");
    pbng_status s = newton_ready(m, p);
    if (s) return s;
    pbng_params q = *p;
    q.resume = 0;
    if ((s = begin(m, u_dev, &q, true))) return s;
    cudaStream_t st = m->stream;
    const int n = m->nfree;
    const State u0 = state_of(m, 0), ut = state_of(m, 3);
    float4* r = (float4*)m->d_nw[0].p;
    float4* x = (float4*)m->d_nw[1].p;
    float4* z = (float4*)m->d_nw[2].p;
    float4* pd = (float4*)m->d_nw[3].p;
    float4* hq = (float4*)m->d_nw[4].p;
    double* sc = (double*)m->d_nw_sc.p;
    int32_t* flag = (int32_t*)m->d_nw_flag.p;
    double* part0 = (double*)m->d_nw_part[0].p;
    double* part1 = (double*)m->d_nw_part[1].p;
    const float4* diag = (const float4*)m->d_diag.p;
    pbng_newton_info nfo{};
    double r0 = 0.0;
    for (double v : m->r0) r0 += v * v;
    r0 = std::sqrt(r0);
    if (!(r0 > 0.0)) r0 = 1.0;
    double rr = 0.0;
    if ((s = newton_force(m, u0, &rr))) return s;
    double rel = std::sqrt(rr) / r0;
    pbng_status result = PBNG_ENOTCONVERGED;
    auto line_search = [&](bool* accepted) -> pbng_status {
        *accepted = false;
        double sl = 1.0;
        for (int t = 0; t < 12 && !*accepted; ++t, sl *= 0.5) {
            PBNG_CUDA(m, launch_newton_axpy(m->nv, n, u0, x, (float)sl, ut, st));
            m->kernel_launches++;
            double rt = 0.0;
            pbng_status e = newton_force(m, ut, &rt);
            if (e) return e;
            if (std::isfinite(rt) && std::sqrt(rt) < (1.0 - 1e-4 * sl) * std::sqrt(rr)) {
                PBNG_CUDA(m, launch_copy_state(m->nv, ut, u0, st));
                m->kernel_launches++;
                rr = rt;
                *accepted = true;
            } else {
                ++nfo.line_search_halvings;
            }
        }
        return PBNG_OK;
    };
    while (rel > rel_tol && nfo.newton_iterations < max_newton) {
        PBNG_CUDA(m, cudaMemsetAsync(pd, 0, sizeof(float4) * (size_t)m->nv, st));
        PBNG_CUDA(m, cudaMemsetAsync(flag, 0, sizeof(int32_t), st));
        PBNG_CUDA(m, launch_cg_init(n, r, diag, x, z, pd, part0, st));
        PBNG_CUDA(m, launch_reduce(part0, vec_blocks(n), sc, st));
        m->kernel_launches += 2;
        const double bnorm = std::sqrt(rr);
        int k = 0;
        while (k < max_cg) {
            PBNG_CUDA(m, launch_adjoint_ring_apply(m->dm, u0, pd, (const Item*)m->d_items.p, m->nitems_ring,
                                                   (int32_t*)m->d_err.p, m->model, hq, part1, st));
            PBNG_CUDA(m, launch_reduce(part1, adjoint_ring_apply_warps(m->nitems_ring), sc + 1, st));
            PBNG_CUDA(m, launch_cg_update(n, sc, x, r, pd, hq, diag, z, part0, part1, flag, st));
            PBNG_CUDA(m, launch_reduce(part0, vec_blocks(n), sc + 2, st));
            PBNG_CUDA(m, launch_reduce(part1, vec_blocks(n), sc + 3, st));
            PBNG_CUDA(m, launch_cg_dir(n, sc, z, pd, flag, sc, st));
            m->kernel_launches += 7;
            ++k;
            if (k % 8 == 0 || k == max_cg) {
                PBNG_CUDA(m, cudaMemcpyAsync(m->h_nw, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
                PBNG_CUDA(m, cudaMemcpyAsync(m->h_nw + 1, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                PBNG_CUDA(m, cudaStreamSynchronize(st));
                int32_t f = 0;
                std::memcpy(&f, m->h_nw + 1, sizeof(int32_t));
                if (f || std::sqrt(m->h_nw[0]) <= cg_tol * bnorm) break;
            }
        }
        nfo.cg_iterations += k;
        if ((s = check_err(m))) return s;
        bool ok = false;
        if ((s = line_search(&ok))) return s;
        if (!ok) {  // fall back to the preconditioned residual at u0 (recomputed: r was overwritten)
            if ((s = newton_force(m, u0, &rr))) return s;
            PBNG_CUDA(m, launch_cg_init(n, r, diag, x, z, pd, part0, st));
            PBNG_CUDA(m, cudaMemcpyAsync(x, z, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToDevice, st));
            m->kernel_launches++;
            ++nfo.fallbacks;
            if ((s = line_search(&ok))) return s;
            if (!ok) {
                // newton_force(ut) ran last: restore r and the blocks at u0
                if ((s = newton_force(m, u0, &rr))) return s;
                ++nfo.newton_iterations;
                m->err = "line search failed";
                break;
            }
        }
        ++nfo.newton_iterations;
        rel = std::sqrt(rr) / r0;
        if (!std::isfinite(rel)) {
            result = PBNG_EDIVERGED;
            break;
        }
    }
    if (rel <= rel_tol) result = PBNG_OK;
    PBNG_CUDA(m, launch_store(m->nv, (const int32_t*)m->d_perm.p, u0, u_dev, st));
    m->kernel_launches++;
    PBNG_CUDA(m, cudaStreamSynchronize(st));
    m->has_state = false;  // the acceleration history does not describe this iterate
    nfo.rel_residual = rel;
    if (info) *info = nfo;
    if (result == PBNG_ENOTCONVERGED && m->err.empty()) m->err = "max Newton iterations reached";
    return result;
}

namespace {
struct StateHeader {
    uint64_t magic;     // "PBNGSTA1"
    int64_t nv, nfree, ncol, ncomp;
    int64_t sweep_l, p1_slot, has_state;
    double omega_l;
    uint64_t perm_hash;
};
constexpr uint64_t kStateMagic = 0x31415453474e4250ull;

uint64_t perm_hash(const std::vector<int32_t>& perm) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the internal order
    for (int32_t v : perm) {
        h ^= (uint64_t)(uint32_t)v;
        h *= 1099511628211ull;
    }
    return h;
}
}  // namespace

pbng_status pbng_get_state(pbng_mesh* m, void* buf, size_t* bytes) {
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if (!bytes) return fail(m, PBNG_EINVAL, "NULL size");
    const size_t arr = sizeof(float4) * (size_t)m->nv;
    const size_t need = sizeof(StateHeader) + sizeof(double) * m->ncomp + 6 * arr;
    if (!buf) {
        *bytes = need;
        return PBNG_OK;
    }
    if (*bytes < need) return fail(m, PBNG_EINVAL, "state buffer too small");
    StateHeader h{kStateMagic, m->nv, m->nfree, m->ncol, m->ncomp, m->sweep_l, m->p1_slot, m->has_state ? 1 : 0,
                  m->omega_l, perm_hash(m->perm)};
    char* out = static_cast<char*>(buf);
    std::memcpy(out, &h, sizeof(h));
    out += sizeof(h);
    for (int k = 0; k < m->ncomp; ++k) {
        const double r = (k < (int)m->r0.size()) ? m->r0[k] : -1.0;
        std::memcpy(out, &r, sizeof(double));
        out += sizeof(double);
    }
    const int slots[3] = {0, m->p1_slot, m->p2_slot};
    for (int sl : slots)
        for (int hl = 0; hl < 2; ++hl) {
            PBNG_CUDA(m, cudaMemcpyAsync(out, m->d_state[sl][hl].p, arr, cudaMemcpyDeviceToHost, m->stream));
            out += arr;
        }
    PBNG_CUDA(m, cudaStreamSynchronize(m->stream));
    *bytes = need;
    return PBNG_OK;
}

pbng_status pbng_set_state(pbng_mesh* m, const void* buf, size_t bytes) {
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if (!buf || bytes < sizeof(StateHeader)) return fail(m, PBNG_EINVAL, "bad state buffer");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    const size_t arr = sizeof(float4) * (size_t)m->nv;
    if (h.magic != kStateMagic || h.nv != m->nv || h.nfree != m->nfree || h.ncol != m->ncol ||
        h.ncomp != m->ncomp || h.perm_hash != perm_hash(m->perm) || (h.p1_slot != 1 && h.p1_slot != 2) ||
        bytes < sizeof(StateHeader) + sizeof(double) * m->ncomp + 6 * arr)
        return fail(m, PBNG_EINVAL, "state does not belong to this mesh layout");
    const char* in = static_cast<const char*>(buf) + sizeof(h);
    m->r0.assign(m->ncomp, -1.0);
    for (int k = 0; k < m->ncomp; ++k) {
        std::memcpy(&m->r0[k], in, sizeof(double));
        in += sizeof(double);
    }
    m->sweep_l = (int32_t)h.sweep_l;
    m->omega_l = h.omega_l;
    m->p1_slot = (int)h.p1_slot;
    m->p2_slot = 3 - m->p1_slot;
    m->has_state = h.has_state != 0;
    const int slots[3] = {0, m->p1_slot, m->p2_slot};
    for (int sl : slots)
        for (int hl = 0; hl < 2; ++hl) {
            PBNG_CUDA(m, cudaMemcpyAsync(m->d_state[sl][hl].p, in, arr, cudaMemcpyHostToDevice, m->stream));
            in += arr;
        }
    PBNG_CUDA(m, cudaStreamSynchronize(m->stream));
    return PBNG_OK;
}

pbng_status pbng_residual(pbng_mesh* m, const float* u_dev, double* residual_out) {
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if (!u_dev || !residual_out) return fail(m, PBNG_EINVAL, "NULL argument");
    PBNG_CUDA(m, launch_load(m->nv, m->nfree, u_dev, (const int32_t*)m->d_perm.p,
                             (const float4*)m->d_dir_hi.p, (const float4*)m->d_dir_lo.p,
                             state_of(m, 3), m->stream));
    m->kernel_launches++;
    std::vector<double> sq(m->ncomp);
    if ((s = residual_sq(m, 3, true, sq.data(), m->all_ring))) return s;
    for (int k = 0; k < m->ncomp; ++k) residual_out[k] = std::sqrt(sq[k]);
    return PBNG_OK;
}

pbng_status pbng_residual_noalloc(pbng_mesh* m, const float* u_dev, double* residual_out) {
    // Same kernels as pbng_residual; the FP64 partial sums go to the fixed
    // scratch array of pbng_kernels.cu instead of handle buffers, and nothing
    // (device or host) is allocated here.
    if (!m) return PBNG_EINVAL;
    m->err.clear();
    if (!u_dev || !residual_out) return fail(m, PBNG_EINVAL, "NULL argument");
    if (m->dirty)
        return fail(m, PBNG_EINVAL,
                    "layout not built: call pbng_get_colouring, pbng_sweep, pbng_solve or "
                    "pbng_residual once after pbng_set_constraints");
    PBNG_CUDA(m, cudaSetDevice(m->device));
    double* scratch = nullptr;
    PBNG_CUDA(m, noalloc_scratch(m->device, &scratch));
    const bool multi = m->ncomp > 1;
    // partial sums (per warp of the ring launch, per block of direct-load
    // colours) then the total, or the per-component sums
    const int64_t nparts = (int64_t)m->ring_partials + m->total_partials;
    const int64_t need = multi ? (int64_t)m->ncomp : nparts + 1;
    if (need > noalloc_scratch_capacity())
        return fail(m, PBNG_EINVAL, "mesh needs more FP64 partial sums than the fixed 65,536-entry scratch holds");
    cudaStream_t st = m->stream;
    PBNG_CUDA(m, launch_load(m->nv, m->nfree, u_dev, (const int32_t*)m->d_perm.p,
                             (const float4*)m->d_dir_hi.p, (const float4*)m->d_dir_lo.p,
                             state_of(m, 3), st));
    // per-component sums accumulate atomically and start at zero (the memset
    // in enqueue_residual); every partial is written before it is summed
    pbng_status r = enqueue_residual(m, state_of(m, 3), true, scratch, scratch, scratch + nparts, st, m->all_ring,
                                     true);
    if (r) return r;
    PBNG_CUDA(m, cudaMemcpyAsync(m->h_pinned, multi ? scratch : scratch + nparts,
                                 sizeof(double) * (multi ? m->ncomp : 1), cudaMemcpyDeviceToHost, st));
    if ((r = sync_with_err(m, st))) return r;
    for (int k = 0; k < m->ncomp; ++k) residual_out[k] = (m->ncol == 0) ? 0.0 : std::sqrt(m->h_pinned[k]);
    return PBNG_OK;
}

pbng_status pbng_test_set_copy_shortfall(pbng_mesh* m, int32_t bytes) {
    if (!m || bytes < 0 || bytes > 1024 || bytes % 16 != 0) return PBNG_EINVAL;
    m->copy_shortfall = bytes;
    m->dm.copy_shortfall = bytes;
    destroy_graphs(m);  // captured launches carry the old value
    return PBNG_OK;
}

pbng_status pbng_set_profiling(pbng_mesh* m, int32_t enable) {
    if (!m) return PBNG_EINVAL;
    m->err.clear();
    PBNG_CUDA(m, prof_flush(m));
    m->prof = enable != 0;
    if (m->prof) {
        for (int k = 0; k < 3; ++k) {
            m->prof_launches[k] = 0;
            m->prof_ms[k] = 0.0;
        }
        m->kernel_launches = 0;
    }
    return PBNG_OK;
}

pbng_status pbng_get_profile(pbng_mesh* m, pbng_profile* out) {
    pbng_status s = ensure_ready(m);
    if (s) return s;
    if (!out) return fail(m, PBNG_EINVAL, "NULL profile");
    PBNG_CUDA(m, prof_flush(m));
    PBNG_CUDA(m, cudaStreamSynchronize(m->stream));
    std::memset(out, 0, sizeof(*out));
    out->colour_pass_launches = m->prof_launches[kProfColour];
    out->colour_pass_ms = m->prof_ms[kProfColour];
    out->accel_launches = m->prof_launches[kProfAccel];
    out->accel_ms = m->prof_ms[kProfAccel];
    out->residual_launches = m->prof_launches[kProfResidual];
    out->residual_ms = m->prof_ms[kProfResidual];
    out->kernel_launches = m->kernel_launches;
    out->free_vertices = m->nfree;
    out->incidences = m->ninc;
    out->ncolours = m->ncol;
    out->colour_ms = m->colour_ms;
    out->layout_ms = m->layout_ms;
    return PBNG_OK;
}

pbng_status pbng_get_schedule(pbng_mesh* m, pbng_schedule* out) {
    if (!m || !out) return PBNG_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->ncolours = m->ncol;
    for (int c = 0; c < std::min<int>(m->ncol, PBNG_MAX_COLOURS); ++c) {
        const bool ring = c < (int)m->ring_colour.size() && m->ring_colour[c];
        out->ctas_per_sm[c] = ring ? m->sched[c].ctas_per_sm : 0;
        out->blocked[c] = ring ? m->sched[c].blocked : 0;
        out->balanced[c] = ring ? m->sched[c].balanced : 0;
    }
    out->default_ms_per_sweep = m->tune_default_ms;
    out->tuned_ms_per_sweep = m->tune_ms;
    out->candidates = m->tune_cands;
    return PBNG_OK;
}

pbng_status pbng_set_schedule(pbng_mesh* m, const pbng_params* p, const pbng_schedule* s) {
    if (!m || !s) return PBNG_EINVAL;
    pbng_params dp;
    if (!p) {
        pbng_default_params(&dp);
        p = &dp;
    }
    if (!valid_params(p)) return fail(m, PBNG_EINVAL, "invalid pbng_params");
    select_path(m, p);
    pbng_status r = ensure_ready(m);
    if (r) return r;
    const int cap = ring_max_ctas_per_sm();
    for (int c = 0; c < std::min<int>(std::min(s->ncolours, m->ncol), PBNG_MAX_COLOURS); ++c) {
        m->sched[c].ctas_per_sm = std::max(1, std::min(cap, (int)s->ctas_per_sm[c]));
        m->sched[c].blocked = s->blocked[c] ? 1 : 0;
        m->sched[c].balanced = s->balanced[c] ? 1 : 0;
    }
    m->tune_default_ms = m->tune_ms = 0.0;
    m->tune_cands = 0;
    destroy_graphs(m);
    return PBNG_OK;
}

// Times every schedule of every ring colour on a scratch copy of u_dev.  One
// timed "round" runs each candidate once over all colours (every colour pass
// of a sweep with that candidate), so the candidates alternate in time and
// share the clock and cache conditions; reps rounds are summed.
pbng_status pbng_autotune(pbng_mesh* m, const float* u_dev, const pbng_params* p, int32_t reps,
                          pbng_schedule* out) {
    if (!m) return PBNG_EINVAL;
    pbng_params dp;
    if (!p) {
        pbng_default_params(&dp);
        p = &dp;
    }
    if (!valid_params(p) || reps < 1 || reps > 1000 || !u_dev) return fail(m, PBNG_EINVAL, "bad autotune arguments");
    select_path(m, p);
    pbng_status r = ensure_ready(m);
    if (r) return r;
    cudaStream_t st = m->stream;
    const bool comp = pair_iterate(p->precision);
    const PassParams pp{(float)p->step, (float)p->skip_tol, p->model};
    const State scratch = state_of(m, 3);
    const int cap = ring_max_ctas_per_sm();
    std::vector<RingSched> cands{{cap, 0, 0}};   // the default first
    for (int cps = 1; cps <= cap; ++cps)
        for (int b = 0; b < 2; ++b)
            for (int bal = 0; bal < 2; ++bal)
                if (!(cps == cap && b == 0 && bal == 0)) cands.push_back({cps, b, bal});
    const int nc = (int)cands.size(), ncol = m->ncol;
    auto pass = [&](int c, RingSched sc) -> pbng_status {
        if (m->ring_colour[c])
            PBNG_CUDA(m, launch_ring_pass(m->dm, scratch, (const Item*)m->d_pitems.p + m->pitem_off[c],
                                          m->pitem_off[c + 1] - m->pitem_off[c], pp, comp, sc,
                                          (int32_t*)m->d_err.p, st));
        else
            PBNG_CUDA(m, launch_colour_pass(m->dm, scratch, m->tables[c], pp, comp, (int32_t*)m->d_err.p, st));
        m->kernel_launches++;
        return PBNG_OK;
    };
    PBNG_CUDA(m, launch_load(m->nv, m->nfree, u_dev, (const int32_t*)m->d_perm.p, (const float4*)m->d_dir_hi.p,
                             (const float4*)m->d_dir_lo.p, scratch, st));
    m->kernel_launches++;
    for (int w = 0; w < 2; ++w)  // warm-up sweeps
        for (int c = 0; c < ncol; ++c)
            if (m->tables[c].total_blocks > 0 && (r = pass(c, cands[0]))) return r;
    std::vector<double> t((size_t)ncol * nc, 0.0);
    std::vector<cudaEvent_t> ev((size_t)2 * ncol * nc, nullptr);
    pbng_status res = PBNG_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            res = fail(m, PBNG_ECUDA, "cudaEventCreate");
            break;
        }
    for (int k = 0; k < reps && res == PBNG_OK; ++k) {
        for (int ci = 0; ci < nc && res == PBNG_OK; ++ci)
            for (int c = 0; c < ncol && res == PBNG_OK; ++c) {
                if (m->tables[c].total_blocks <= 0) continue;
                cudaEvent_t* e = &ev[2 * ((size_t)ci * ncol + c)];
                if (cudaEventRecord(e[0], st) != cudaSuccess) res = fail(m, PBNG_ECUDA, "cudaEventRecord");
                if (res == PBNG_OK) res = pass(c, m->ring_colour[c] ? cands[ci] : cands[0]);
                if (res == PBNG_OK && cudaEventRecord(e[1], st) != cudaSuccess)
                    res = fail(m, PBNG_ECUDA, "cudaEventRecord");
            }
        if (res == PBNG_OK && cudaStreamSynchronize(st) != cudaSuccess) res = fail(m, PBNG_ECUDA, "synchronize");
        for (int ci = 0; ci < nc && res == PBNG_OK; ++ci)
            for (int c = 0; c < ncol; ++c) {
                if (m->tables[c].total_blocks <= 0) continue;
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, ev[2 * ((size_t)ci * ncol + c)], ev[2 * ((size_t)ci * ncol + c) + 1]) !=
                    cudaSuccess) {
                    res = fail(m, PBNG_ECUDA, "cudaEventElapsedTime");
                    break;
                }
                t[(size_t)c * nc + ci] += ms;
            }
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (res) return res;
    if ((r = check_err(m))) return r;
    double t_def = 0.0, t_new = 0.0;
    for (int c = 0; c < ncol; ++c) {
        int best = 0;
        if (m->ring_colour[c])
            for (int ci = 1; ci < nc; ++ci)
                if (t[(size_t)c * nc + ci] < t[(size_t)c * nc + best]) best = ci;
        if (t[(size_t)c * nc + best] > 0.98 * t[(size_t)c * nc]) best = 0;
        m->sched[c] = cands[best];
        t_def += t[(size_t)c * nc];
        t_new += t[(size_t)c * nc + best];
    }
    destroy_graphs(m);
    m->tune_default_ms = t_def / reps;
    m->tune_ms = t_new / reps;
    m->tune_cands = nc;
    return out ? pbng_get_schedule(m, out) : PBNG_OK;
}

pbng_status pbng_get_solve_info(const pbng_mesh* m, pbng_solve_info* out) {
    if (!m || !out) return PBNG_EINVAL;
    *out = m->info;
    return PBNG_OK;
}

int32_t pbng_num_components(const pbng_mesh* m) { return m ? m->ncomp : 0; }

pbng_status pbng_measure_fp32_peak(void* stream, double* tflops_out) {
    if (!tflops_out) return PBNG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return PBNG_ECUDA;
    const int blocks = nsm * 8;  // 2048 threads per SM
    float* out = nullptr;
    if (cudaMalloc((void**)&out, sizeof(float) * 256 * (size_t)blocks) != cudaSuccess) return PBNG_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pbng_status r = PBNG_OK;
    double best = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = PBNG_ECUDA;
    for (int rep = 0; rep < 6 && r == PBNG_OK; ++rep) {  // the first launch warms up
        double flops = 0.0;
        float ms = 0.0f;
        if (pbng::fma_peak(st, out, blocks, 1 << 15, e0, e1, &flops) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            r = PBNG_ECUDA;
            break;
        }
        if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (r == PBNG_OK) *tflops_out = best;
    return r;
}

const char* pbng_status_string(pbng_status s) {
    switch (s) {
        case PBNG_OK: return "ok";
        case PBNG_EINVAL: return "invalid argument";
        case PBNG_ENOMEM: return "out of memory";
        case PBNG_ECUDA: return "CUDA error";
        case PBNG_EDEGENERATE: return "degenerate element or nodal Hessian";
        case PBNG_EDIVERGED: return "diverged";
        case PBNG_ETIMEOUT: return "device wait timed out";
        case PBNG_ENOTCONVERGED: return "not converged";
    }
    return "unknown status";
}

const char* pbng_last_error(const pbng_mesh* m) { return m ? m->err.c_str() : ""; }

void pbng_destroy(pbng_mesh* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    DevBuf* bufs[] = {&m->d_lam[0], &m->d_lam[1], &m->d_lam[2], &m->d_gv, &m->d_diag, &m->d_hdl, &m->d_tv,
                      &m->d_tb, &m->d_dq_int, &m->d_dq_caller, &m->d_adj_partial,
                      &m->d_inc_off, &m->d_rec_a, &m->d_rec_b, &m->d_rec_c, &m->d_rec_d,
                      &m->d_ring, &m->d_ring_lo, &m->d_items, &m->d_prec, &m->d_pids, &m->d_pitems, &m->d_host_u, &m->d_vsq, &m->d_comp_off,
                      &m->d_comp_list, &m->d_lam_hi, &m->d_lam_lo, &m->d_rhs, &m->d_fp[0], &m->d_fp[1], &m->d_fp[2],
                      &m->d_fp[3], &m->d_shift[0][0], &m->d_shift[0][1], &m->d_shift[1][0], &m->d_shift[1][1],
                      &m->d_maxabs, &m->d_refine_partial, &m->d_acg[0], &m->d_acg[1], &m->d_acg_part[0],
                      &m->d_acg_part[1], &m->d_acg_sc,
                      &m->d_aux0, &m->d_aux1, &m->d_aux_lo, &m->d_comp, &m->d_perm, &m->d_dir_hi, &m->d_dir_lo,
                      &m->d_aux_base0, &m->d_aux_base1, &m->d_be_k, &m->d_wc_off, &m->d_wc_list, &m->d_wc_v,
                      &m->d_wc_b, &m->d_wc_k, &m->d_wc_c0,
                      &m->d_nw[0], &m->d_nw[1], &m->d_nw[2], &m->d_nw[3], &m->d_nw[4], &m->d_nw_part[0],
                      &m->d_nw_part[1], &m->d_nw_sc, &m->d_nw_flag,
                      &m->d_partial, &m->d_comp_sq, &m->d_scalar, &m->d_err};
    for (DevBuf* b : bufs) free_buf(*b);
    for (auto& sb : m->d_state)
        for (auto& b : sb) free_buf(b);
    for (auto& p : m->ev_used) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : m->ev_free) cudaEventDestroy(e);
    destroy_graphs(m);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    if (m->h_wg) cudaFreeHost(m->h_wg);
    free_buf(m->d_wg);
    if (m->h_pinned) cudaFreeHost(m->h_pinned);
    if (m->h_active) cudaFreeHost(m->h_active);
    if (m->h_nw) cudaFreeHost(m->h_nw);
    free_buf(m->d_active);
    delete m;
}

}  // extern "C"
