// Host build of the extended-precision element force (the __host__ side of
// paper_2306_09021_gb300/csrc/pbng_ff.cuh) for tests/test_ff_host.py, which
// compares it with the FP64 oracle on the CPU.  Inputs are doubles; each is
// split into the float pair (hi, lo) that the extended passes store.
#include "pbng_ff.cuh"

namespace {
pbng::ff::F2 split(double x) {
    const float h = (float)x;
    return pbng::ff::mk(h, (float)(x - (double)h));
}
}  // namespace

// g: dN/dX of the three other vertices (3x3, row k = vertex k); d: their
// displacements relative to the vertex (3x3, row k); a = 2 mu V, b = lambda V;
// q: float32 quaternion (w, x, y, z) of the polar rotation (corotated only);
// out: V P(F) s with s = g_1 + g_2 + g_3, as hi + lo in double.
extern "C" int ff_element_force(int model, const double* g, const double* d, double a, double b, const float* q,
                                double* out) {
    pbng::ff::F2 gg[3][3], dd[3][3], f[3];
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) {
            gg[k][c] = split(g[3 * k + c]);
            dd[k][c] = split(d[3 * k + c]);
        }
    const pbng::ff::F2 a2 = split(a), b2 = split(b);
    switch (model) {
        case 0: pbng::ff::element_force<0>(gg, a2, b2, dd, q, f); break;
        case 1: pbng::ff::element_force<1>(gg, a2, b2, dd, q, f); break;
        case 2: pbng::ff::element_force<2>(gg, a2, b2, dd, q, f); break;
        default: return -1;
    }
    for (int p = 0; p < 3; ++p) out[p] = (double)f[p].h + (double)f[p].l;
    return 0;
}
