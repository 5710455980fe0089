// PBNG FP64 oracle — TEST INFRASTRUCTURE ONLY (see pbng_oracle.h).
//
// Plain, serial restatement of the paper's method in double precision.  Every
// function cites the passage it follows.  No blocking, fusion or reordering
// beyond what the paper states; nothing here is shared with the CUDA library.

#include "pbng_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <array>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- 3x3 algebra
void mat_mul(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

void mat_mul_tn(const double* A, const double* B, double* C) {  // A^T B
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * k + i] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

void mat_mul_nt(const double* A, const double* B, double* C) {  // A B^T
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * j + k];
            C[3 * i + j] = s;
        }
}

double det3(const double* F) {
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

// Cofactor matrix: row i is the cross product of the other two rows (cyclic),
// equal to det(F) F^{-T} when F is invertible and defined for every F.
void cof3(const double* F, double* C) {
    C[0] = F[4] * F[8] - F[5] * F[7];
    C[1] = F[5] * F[6] - F[3] * F[8];
    C[2] = F[3] * F[7] - F[4] * F[6];
    C[3] = F[7] * F[2] - F[8] * F[1];
    C[4] = F[8] * F[0] - F[6] * F[2];
    C[5] = F[6] * F[1] - F[7] * F[0];
    C[6] = F[1] * F[5] - F[2] * F[4];
    C[7] = F[2] * F[3] - F[0] * F[5];
    C[8] = F[0] * F[4] - F[1] * F[3];
}

void mat_vec(const double* A, const double* v, double* out) {
    for (int i = 0; i < 3; ++i) out[i] = A[3 * i] * v[0] + A[3 * i + 1] * v[1] + A[3 * i + 2] * v[2];
}

void cross(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Solve A d = r for SPD 3x3 A by Cholesky.  Returns false if A is not SPD.
bool chol_solve3(const double* A, const double* r, double* d) {
    double L[9] = {0};
    for (int j = 0; j < 3; ++j) {
        double s = A[3 * j + j];
        for (int k = 0; k < j; ++k) s -= L[3 * j + k] * L[3 * j + k];
        if (!(s > 0.0)) return false;
        L[3 * j + j] = std::sqrt(s);
        for (int i = j + 1; i < 3; ++i) {
            double t = A[3 * i + j];
            for (int k = 0; k < j; ++k) t -= L[3 * i + k] * L[3 * j + k];
            L[3 * i + j] = t / L[3 * j + j];
        }
    }
    double y[3];
    for (int i = 0; i < 3; ++i) {
        double t = r[i];
        for (int k = 0; k < i; ++k) t -= L[3 * i + k] * y[k];
        y[i] = t / L[3 * i + i];
    }
    for (int i = 2; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < 3; ++k) t -= L[3 * k + i] * d[k];
        d[i] = t / L[3 * i + i];
    }
    return true;
}

// Dense LU with partial pivoting; solves A x = b in place (A n x n row-major).
bool lu_solve(std::vector<double> A, std::vector<double>& b, int n) {
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = std::fabs(A[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0) return false;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
            std::swap(b[k], b[p]);
        }
        for (int i = k + 1; i < n; ++i) {
            double m = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            if (m == 0.0) continue;
            for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= m * A[(size_t)k * n + j];
            b[i] -= m * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = b[i];
        for (int j = i + 1; j < n; ++j) t -= A[(size_t)i * n + j] * b[j];
        b[i] = t / A[(size_t)i * n + i];
    }
    return true;
}

// --------------------------------------------------- SVD and polar rotation
// One-sided Jacobi (Hestenes): rotate column pairs of A = F V until they are
// mutually orthogonal; then s_j = |A_j| and U_j = A_j / s_j.
int svd3(const double* F, double* U, double* s, double* V) {
    double A[9];
    std::memcpy(A, F, sizeof(A));
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    int sweeps = 0;
    for (; sweeps < 100; ++sweeps) {
        bool rotated = false;
        for (const auto& pq : P) {
            int p = pq[0], q = pq[1];
            double al = 0, be = 0, ga = 0;
            for (int i = 0; i < 3; ++i) {
                al += A[3 * i + p] * A[3 * i + p];
                be += A[3 * i + q] * A[3 * i + q];
                ga += A[3 * i + p] * A[3 * i + q];
            }
            if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
            rotated = true;
            double zeta = (be - al) / (2.0 * ga);
            double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
            double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
            for (int i = 0; i < 3; ++i) {
                double ap = A[3 * i + p], aq = A[3 * i + q];
                A[3 * i + p] = c * ap - sn * aq;
                A[3 * i + q] = sn * ap + c * aq;
                double vp = V[3 * i + p], vq = V[3 * i + q];
                V[3 * i + p] = c * vp - sn * vq;
                V[3 * i + q] = sn * vp + c * vq;
            }
        }
        if (!rotated) break;
    }
    double sig[3];
    for (int j = 0; j < 3; ++j)
        sig[j] = std::sqrt(A[j] * A[j] + A[3 + j] * A[3 + j] + A[6 + j] * A[6 + j]);
    int ord[3] = {0, 1, 2};
    std::stable_sort(ord, ord + 3, [&](int a, int b) { return sig[a] > sig[b]; });
    double Vs[9], As[9];
    for (int jj = 0; jj < 3; ++jj) {
        int j = ord[jj];
        s[jj] = sig[j];
        for (int i = 0; i < 3; ++i) {
            Vs[3 * i + jj] = V[3 * i + j];
            As[3 * i + jj] = A[3 * i + j];
        }
    }
    std::memcpy(V, Vs, sizeof(Vs));
    // Left vectors; complete by cross products where a singular value vanishes.
    double tiny = 1e-13 * (s[0] > 0 ? s[0] : 1.0);
    double u[3][3];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) u[j][i] = (s[j] > tiny) ? As[3 * i + j] / s[j] : 0.0;
    if (!(s[0] > tiny)) { u[0][0] = 1; u[0][1] = 0; u[0][2] = 0; }
    if (!(s[1] > tiny)) {
        double e[3] = {0, 0, 0};
        e[std::fabs(u[0][0]) < 0.9 ? 0 : 1] = 1.0;
        cross(u[0], e, u[1]);
        double n = std::sqrt(u[1][0] * u[1][0] + u[1][1] * u[1][1] + u[1][2] * u[1][2]);
        for (int i = 0; i < 3; ++i) u[1][i] /= n;
    }
    if (!(s[2] > tiny)) cross(u[0], u[1], u[2]);
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) U[3 * i + j] = u[j][i];
    return sweeps;
}

// Section "Constitutive Models" (Eq. cor) with the rotation R of F = RS taken
// in SO(3): the smallest singular value carries the sign of det F.
void polar(const double* F, double* R, double* shat) {
    double U[9], s[3], V[9];
    svd3(F, U, s, V);
    double sg = (det3(U) * det3(V) < 0.0) ? -1.0 : 1.0;
    double UD[9];
    std::memcpy(UD, U, sizeof(UD));
    for (int i = 0; i < 3; ++i) UD[3 * i + 2] *= sg;
    mat_mul_nt(UD, V, R);
    if (shat) { shat[0] = s[0]; shat[1] = s[1]; shat[2] = sg * s[2]; }
}

// Models of Section "Constitutive Models": 0 corotated (Eq. cor), 1
// Neo-Hookean in the Macklin-Mueller form (Eq. nh, lambda_hat = mu + lambda),
// 2 stable Neo-Hookean (Eq. snh).  The printed Eq. snh has no lambda on its
// volume term; it is read as Smith et al.'s (lambda/2)(J - alpha)^2 with
// alpha = 1 + 3 mu'/(4 lambda'), and, as Section "Lame Coefficients"
// requires of a model set from Lame coefficients, its Hessian at F = I is
// made equal to linear elasticity's by Smith et al.'s mu' = 4 mu / 3,
// lambda' = lambda + 5 mu / 6.
enum { kCorotated = 0, kNeoHookean = 1, kStableNeoHookean = 2 };

void snh_params(double mu, double lam, double* mus, double* lams, double* alpha) {
    *mus = 4.0 * mu / 3.0;
    *lams = lam + 5.0 * mu / 6.0;
    *alpha = 1.0 + 3.0 * (*mus) / (4.0 * (*lams));
}

double frob2(const double* F) {
    double n2 = 0.0;
    for (int i = 0; i < 9; ++i) n2 += F[i] * F[i];
    return n2;
}

double psi(const double* F, double mu, double lam, int model) {
    const double J = det3(F);
    if (model == kNeoHookean) {  // Eq. nh
        const double lh = mu + lam, c = J - 1.0 - mu / lh;
        return 0.5 * mu * frob2(F) + 0.5 * lh * c * c;
    }
    if (model == kStableNeoHookean) {  // Eq. snh
        double mus, lams, alpha;
        snh_params(mu, lam, &mus, &lams, &alpha);
        const double ic = frob2(F);
        return 0.5 * mus * (ic - 3.0) + 0.5 * lams * (J - alpha) * (J - alpha) - 0.5 * mus * std::log(1.0 + ic);
    }
    double R[9];  // Eq. cor
    polar(F, R, nullptr);
    double n2 = 0.0;
    for (int i = 0; i < 9; ++i) n2 += (F[i] - R[i]) * (F[i] - R[i]);
    return mu * n2 + 0.5 * lam * (J - 1.0) * (J - 1.0);
}

// P = dPsi/dF.  With C = cof F = dJ/dF:
//   corotated  2 mu (F - R) + lambda (J - 1) C
//   NH         mu F + lambda_hat (J - 1 - mu / lambda_hat) C
//   SNH        mu' (1 - 1 / (1 + |F|^2)) F + lambda' (J - alpha) C
void pk1(const double* F, double mu, double lam, int model, double* P) {
    double C[9];
    cof3(F, C);
    const double J = det3(F);
    if (model == kNeoHookean) {
        const double lh = mu + lam, k = lh * (J - 1.0 - mu / lh);
        for (int i = 0; i < 9; ++i) P[i] = mu * F[i] + k * C[i];
        return;
    }
    if (model == kStableNeoHookean) {
        double mus, lams, alpha;
        snh_params(mu, lam, &mus, &lams, &alpha);
        const double s = mus * (1.0 - 1.0 / (1.0 + frob2(F))), k = lams * (J - alpha);
        for (int i = 0; i < 9; ++i) P[i] = s * F[i] + k * C[i];
        return;
    }
    double R[9];
    polar(F, R, nullptr);
    for (int i = 0; i < 9; ++i) P[i] = 2.0 * mu * (F[i] - R[i]) + lam * (J - 1.0) * C[i];
}

// The bilinear part dC of F -> cof F in direction dF: cof(F + dF) - cof F - cof dF.
void dcof3(const double* F, const double* dF, double* dC) {
    double Fp[9], Cp[9], C[9], Cd[9];
    for (int i = 0; i < 9; ++i) Fp[i] = F[i] + dF[i];
    cof3(Fp, Cp);
    cof3(F, C);
    cof3(dF, Cd);
    for (int i = 0; i < 9; ++i) dC[i] = Cp[i] - C[i] - Cd[i];
}

// dP = (d^2 Psi / dF^2) : dF (the density Hessian of Eq. hess).
//   corotated  2mu(dF - dR) + lam (C:dF) C + lam (J-1) dC, dR = R [w]_x with
//              (tr S I - S) w = axial(R^T dF - dF^T R), S = R^T F
//   NH         mu dF + lambda_hat (C:dF) C + lambda_hat (J - 1 - mu/lambda_hat) dC
//   SNH        mu' (1 - 1/(1+|F|^2)) dF + mu' 2 (F:dF) / (1+|F|^2)^2 F
//              + lambda' (C:dF) C + lambda' (J - alpha) dC
void dpk1(const double* F, const double* dF, double mu, double lam, int model, double* dP) {
    if (model == kNeoHookean || model == kStableNeoHookean) {
        double C[9], dC[9];
        cof3(F, C);
        dcof3(F, dF, dC);
        const double J = det3(F);
        double CdF = 0.0, FdF = 0.0;
        for (int i = 0; i < 9; ++i) {
            CdF += C[i] * dF[i];
            FdF += F[i] * dF[i];
        }
        if (model == kNeoHookean) {
            const double lh = mu + lam, k = lh * (J - 1.0 - mu / lh);
            for (int i = 0; i < 9; ++i) dP[i] = mu * dF[i] + lh * CdF * C[i] + k * dC[i];
        } else {
            double mus, lams, alpha;
            snh_params(mu, lam, &mus, &lams, &alpha);
            const double q = 1.0 + frob2(F);
            const double s = mus * (1.0 - 1.0 / q), t = mus * 2.0 * FdF / (q * q), k = lams * (J - alpha);
            for (int i = 0; i < 9; ++i) dP[i] = s * dF[i] + t * F[i] + lams * CdF * C[i] + k * dC[i];
        }
        return;
    }
    double R[9], S[9], RtdF[9];
    polar(F, R, nullptr);
    mat_mul_tn(R, F, S);
    mat_mul_tn(R, dF, RtdF);
    double rhs[3] = {RtdF[7] - RtdF[5], RtdF[2] - RtdF[6], RtdF[3] - RtdF[1]};
    double trS = S[0] + S[4] + S[8];
    double M[9];
    for (int i = 0; i < 9; ++i) M[i] = -0.5 * (S[i] + S[(i % 3) * 3 + i / 3]);
    M[0] += trS; M[4] += trS; M[8] += trS;
    std::vector<double> Mv(M, M + 9), b(rhs, rhs + 3);
    double w[3] = {0, 0, 0};
    if (lu_solve(Mv, b, 3)) { w[0] = b[0]; w[1] = b[1]; w[2] = b[2]; }
    double W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double dR[9];
    mat_mul(R, W, dR);
    double C[9], Cp[9], Cd[9], Fp[9];
    cof3(F, C);
    for (int i = 0; i < 9; ++i) Fp[i] = F[i] + dF[i];
    cof3(Fp, Cp);
    cof3(dF, Cd);
    double CdF = 0.0;
    for (int i = 0; i < 9; ++i) CdF += C[i] * dF[i];
    double J = det3(F);
    for (int i = 0; i < 9; ++i) {
        double dC = Cp[i] - C[i] - Cd[i];
        dP[i] = 2.0 * mu * (dF[i] - dR[i]) + lam * CdF * C[i] + lam * (J - 1.0) * dC;
    }
}

// ------------------------------------------------------------------- mesh
struct Mesh {
    int nv = 0, ne = 0;
    std::vector<double> X;                 // 3 nv rest positions
    std::vector<int> tets;                 // 4 ne
    std::vector<double> mu, lam, vol, B;   // per tet; B = Dm^{-1}, 9 per tet
    std::vector<unsigned char> dir;        // nv
    std::vector<double> fext;              // 3 nv
    std::vector<int> inc_off, inc_tet, inc_loc;  // vertex -> (tet, local index)
    std::vector<int> spr_off, spr_list;    // vertex -> spring ids
    std::vector<double> spr_t, spr_k;
    bool has_plane = false;
    double pn[3] = {0, 0, 1}, pd = 0.0, kc = 0.0;
    int model = kCorotated;                // Section "Constitutive Models"
    // Backward Euler (Eq. fem_be): lumped masses m_ii and 1/dt^2 (0 = quasistatic),
    // and the inertial target xhat = 2 x^n - x^{n-1}.
    std::vector<double> mass, xhat;
    double inv_dt2 = 0.0;
    // General weak constraints of Section "Weak Constraints":
    // C_c(y) = sum_j (w0_cj - w1_cj) y_j, energy (1/2) C^T K_c C,
    // K_c = k_tau I + (k_n - k_tau) n n^T.  wc_v / wc_b hold each constraint's
    // vertices and coefficients w0 - w1 (duplicates merged); vert_wc lists the
    // constraints of every vertex.
    std::vector<std::vector<int>> wc_v;
    std::vector<std::vector<double>> wc_b;
    std::vector<std::array<double, 9>> wc_K;
    std::vector<std::vector<int>> vert_wc;
    std::vector<int> colour;               // nv, -1 clamped
    std::vector<std::vector<int>> by_colour;
    // Order of the colour passes in one sweep: 0 = ascending (one
    // Gauss-Seidel pass, 0..C-1); 1 = symmetric (0..C-1, then C-2..0).
    int colour_order = 0;
};

// g_j = dN_j/dX in tet e: rows of B for j = 1..3, g_0 = -(g_1 + g_2 + g_3).
void grad(const Mesh& m, int e, int j, double* g) {
    const double* B = &m.B[9 * (size_t)e];
    if (j > 0) {
        for (int a = 0; a < 3; ++a) g[a] = B[3 * (j - 1) + a];
    } else {
        for (int a = 0; a < 3; ++a) g[a] = -(B[a] + B[3 + a] + B[6 + a]);
    }
}

// F = sum_j x_j g_j^T (Eq. disc_pe: the deformation gradient of a P1 tet).
void deformation_gradient(const Mesh& m, const double* x, int e, double* F) {
    for (int i = 0; i < 9; ++i) F[i] = 0.0;
    for (int j = 0; j < 4; ++j) {
        double g[3];
        grad(m, e, j, g);
        const double* xj = &x[3 * (size_t)m.tets[4 * (size_t)e + j]];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) F[3 * a + b] += xj[a] * g[b];
    }
}

// Section "Coloring and Parallelism": visit free nodes in ascending id; a node
// takes the least colour absent from the used-colour sets S_c of every
// element (and multi-node weak constraint; none here) it belongs to, then
// registers that colour in each of those sets.
void group_by_colour(Mesh& m) {
    int ncol = 0;
    for (int i = 0; i < m.nv; ++i) ncol = std::max(ncol, m.colour[i] + 1);
    m.by_colour.assign(ncol, {});
    for (int i = 0; i < m.nv; ++i)
        if (m.colour[i] >= 0) m.by_colour[m.colour[i]].push_back(i);
}

void colour_nodes(Mesh& m) {
    // S_e for tets (first ne sets) and for multi-node weak constraints.
    std::vector<std::set<int>> S(m.ne + m.wc_v.size());
    m.colour.assign(m.nv, -1);
    for (int i = 0; i < m.nv; ++i) {
        if (m.dir[i]) continue;
        std::set<int> used;
        for (int k = m.inc_off[i]; k < m.inc_off[i + 1]; ++k)
            used.insert(S[m.inc_tet[k]].begin(), S[m.inc_tet[k]].end());
        for (int c : m.vert_wc[i]) used.insert(S[m.ne + c].begin(), S[m.ne + c].end());
        int c = 0;
        while (used.count(c)) ++c;
        m.colour[i] = c;
        for (int k = m.inc_off[i]; k < m.inc_off[i + 1]; ++k) S[m.inc_tet[k]].insert(c);
        for (int cc : m.vert_wc[i]) S[m.ne + cc].insert(c);
    }
    group_by_colour(m);
}

// Section "Collision Coloring": only nodes incident to weak constraints are
// revisited (ascending id); each keeps its previous colour unless a node it
// shares a tet or a constraint with already uses it, else takes the least
// colour none of them uses.  Nodes of unchanged constraints keep their
// colours, so visiting all constraint nodes recolours exactly those of the
// new ones.
void recolour_constraint_nodes(Mesh& m) {
    for (int i = 0; i < m.nv; ++i) {
        if (m.dir[i] || m.vert_wc[i].empty()) continue;
        std::set<int> used;
        for (int k = m.inc_off[i]; k < m.inc_off[i + 1]; ++k) {
            const int e = m.inc_tet[k];
            for (int j = 0; j < 4; ++j) {
                const int v = m.tets[4 * (size_t)e + j];
                if (v != i && m.colour[v] >= 0) used.insert(m.colour[v]);
            }
        }
        for (int c : m.vert_wc[i])
            for (int v : m.wc_v[c])
                if (v != i && m.colour[v] >= 0) used.insert(m.colour[v]);
        if (m.colour[i] >= 0 && !used.count(m.colour[i])) continue;
        int c = 0;
        while (used.count(c)) ++c;
        m.colour[i] = c;
    }
    group_by_colour(m);
}

// C_c(x) and the force / Hessian contributions of constraint c on node i.
void wc_value(const Mesh& m, int c, const double* x, double* C) {
    C[0] = C[1] = C[2] = 0.0;
    for (size_t k = 0; k < m.wc_v[c].size(); ++k)
        for (int a = 0; a < 3; ++a) C[a] += m.wc_b[c][k] * x[3 * (size_t)m.wc_v[c][k] + a];
}

double wc_coeff(const Mesh& m, int c, int i) {
    for (size_t k = 0; k < m.wc_v[c].size(); ++k)
        if (m.wc_v[c][k] == i) return m.wc_b[c][k];
    return 0.0;
}

// Right-hand side and modified Hessian of node i (Eq. pbgn_dx with the force
// of Section "Modified Hessian" and A_i of Eq. mod_hess), weak terms included.
void local_system(const Mesh& m, const double* x, int i, double* r, double* A) {
    for (int a = 0; a < 3; ++a) r[a] = m.fext[3 * (size_t)i + a];
    for (int a = 0; a < 9; ++a) A[a] = 0.0;
    for (int k = m.inc_off[i]; k < m.inc_off[i + 1]; ++k) {
        int e = m.inc_tet[k];
        double F[9], P[9], C[9], g[3], Pg[3], w[3];
        deformation_gradient(m, x, e, F);
        pk1(F, m.mu[e], m.lam[e], m.model, P);
        cof3(F, C);
        grad(m, e, m.inc_loc[k], g);
        mat_vec(P, g, Pg);
        mat_vec(C, g, w);
        double V = m.vol[e], gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        for (int a = 0; a < 3; ++a) {
            r[a] -= V * Pg[a];
            A[4 * a] += V * 2.0 * m.mu[e] * gg;
            for (int b = 0; b < 3; ++b) A[3 * a + b] += V * m.lam[e] * w[a] * w[b];
        }
    }
    // Weak constraints of Section "Weak Constraints": a spring to a fixed
    // target (C = x_i - t, K = k I) and plane contact (K = k_n n n^T, k_tau = 0).
    for (int k = m.spr_off[i]; k < m.spr_off[i + 1]; ++k) {
        int s = m.spr_list[k];
        double ks = m.spr_k[s];
        for (int a = 0; a < 3; ++a) {
            r[a] -= ks * (x[3 * (size_t)i + a] - m.spr_t[3 * (size_t)s + a]);
            A[4 * a] += ks;
        }
    }
    if (m.has_plane) {
        const double* xi = &x[3 * (size_t)i];
        double sd = m.pn[0] * xi[0] + m.pn[1] * xi[1] + m.pn[2] * xi[2] - m.pd;
        if (sd < 0.0) {
            for (int a = 0; a < 3; ++a) {
                r[a] -= m.kc * sd * m.pn[a];
                for (int b = 0; b < 3; ++b) A[3 * a + b] += m.kc * m.pn[a] * m.pn[b];
            }
        }
    }
    // General weak constraints: -dE/dx_i = -b_i K C, and b_i^2 K on A
    // (the second term of Eq. mod_hess).
    for (int c : m.vert_wc[i]) {
        double C[3];
        wc_value(m, c, x, C);
        const double b = wc_coeff(m, c, i);
        const double* K = m.wc_K[c].data();
        for (int a = 0; a < 3; ++a) {
            r[a] -= b * (K[3 * a] * C[0] + K[3 * a + 1] * C[1] + K[3 * a + 2] * C[2]);
            for (int bb = 0; bb < 3; ++bb) A[3 * a + bb] += b * b * K[3 * a + bb];
        }
    }
    // Eq. fem_be moved to the right-hand side: -m_ii (x_i - xhat_i) / dt^2,
    // whose derivative adds m_ii / dt^2 to the diagonal of A.
    if (m.inv_dt2 > 0.0) {
        const double k = m.mass[i] * m.inv_dt2;
        for (int a = 0; a < 3; ++a) {
            r[a] -= k * (x[3 * (size_t)i + a] - m.xhat[3 * (size_t)i + a]);
            A[4 * a] += k;
        }
    }
}

// Eq. pbgn_update / pbgn_dx: one modified-Newton step from Delta = 0.
bool node_update(const Mesh& m, double* x, int i, double skip_tol) {
    double r[3], A[9], d[3];
    local_system(m, x, i, r, A);
    if (skip_tol > 0.0 && std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) <= skip_tol) return true;
    if (!chol_solve3(A, r, d)) return false;
    for (int a = 0; a < 3; ++a) x[3 * (size_t)i + a] += d[a];
    return std::isfinite(x[3 * (size_t)i]) && std::isfinite(x[3 * (size_t)i + 1]) &&
           std::isfinite(x[3 * (size_t)i + 2]);
}

double residual(const Mesh& m, const double* x, double* rout) {
    double s = 0.0;
    for (int i = 0; i < m.nv; ++i) {
        double r[3] = {0, 0, 0}, A[9];
        if (!m.dir[i]) local_system(m, x, i, r, A);
        if (rout)
            for (int a = 0; a < 3; ++a) rout[3 * (size_t)i + a] = r[a];
        s += r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    }
    return std::sqrt(s);
}

double energy(const Mesh& m, const double* x) {
    double E = 0.0;
    for (int e = 0; e < m.ne; ++e) {
        double F[9];
        deformation_gradient(m, x, e, F);
        E += m.vol[e] * psi(F, m.mu[e], m.lam[e], m.model);
    }
    for (int i = 0; i < m.nv; ++i) {
        const double* xi = &x[3 * (size_t)i];
        for (int k = m.spr_off[i]; k < m.spr_off[i + 1]; ++k) {
            int s = m.spr_list[k];
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double d = xi[a] - m.spr_t[3 * (size_t)s + a];
                d2 += d * d;
            }
            E += 0.5 * m.spr_k[s] * d2;
        }
        if (m.has_plane) {
            double sd = m.pn[0] * xi[0] + m.pn[1] * xi[1] + m.pn[2] * xi[2] - m.pd;
            if (sd < 0.0) E += 0.5 * m.kc * sd * sd;
        }
        for (int a = 0; a < 3; ++a) E -= m.fext[3 * (size_t)i + a] * xi[a];
        if (m.inv_dt2 > 0.0 && !m.dir[i]) {  // incremental potential of Eq. fem_be
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double d = xi[a] - m.xhat[3 * (size_t)i + a];
                d2 += d * d;
            }
            E += 0.5 * m.mass[i] * m.inv_dt2 * d2;
        }
    }
    for (size_t c = 0; c < m.wc_v.size(); ++c) {  // (1/2) C^T K C
        double C[3];
        wc_value(m, (int)c, x, C);
        const double* K = m.wc_K[c].data();
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) E += 0.5 * C[a] * K[3 * a + b] * C[b];
    }
    return E;
}

// Dense -d(f + f^ext)/dx: the element part assembled from the true density
// Hessian (Eq. hess) one unit direction at a time, plus the weak terms.
void hessian_dense(const Mesh& m, const double* x, std::vector<double>& H) {
    const int n = 3 * m.nv;
    H.assign((size_t)n * n, 0.0);
    for (int e = 0; e < m.ne; ++e) {
        double F[9], g[4][3];
        deformation_gradient(m, x, e, F);
        for (int j = 0; j < 4; ++j) grad(m, e, j, g[j]);
        for (int jb = 0; jb < 4; ++jb)
            for (int b = 0; b < 3; ++b) {
                double dF[9] = {0}, dP[9];
                for (int c = 0; c < 3; ++c) dF[3 * b + c] = g[jb][c];
                dpk1(F, dF, m.mu[e], m.lam[e], m.model, dP);
                int col = 3 * m.tets[4 * (size_t)e + jb] + b;
                for (int ja = 0; ja < 4; ++ja) {
                    double v[3];
                    mat_vec(dP, g[ja], v);
                    int row = 3 * m.tets[4 * (size_t)e + ja];
                    for (int a = 0; a < 3; ++a) H[(size_t)(row + a) * n + col] += m.vol[e] * v[a];
                }
            }
    }
    for (size_t c = 0; c < m.wc_v.size(); ++c)
        for (size_t p = 0; p < m.wc_v[c].size(); ++p)
            for (size_t q = 0; q < m.wc_v[c].size(); ++q) {
                const int vi = m.wc_v[c][p], vj = m.wc_v[c][q];
                const double bb = m.wc_b[c][p] * m.wc_b[c][q];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        H[(size_t)(3 * vi + a) * n + 3 * vj + b] += bb * m.wc_K[c][3 * a + b];
            }
    for (int i = 0; i < m.nv; ++i) {
        const double* xi = &x[3 * (size_t)i];
        if (m.inv_dt2 > 0.0 && !m.dir[i])
            for (int a = 0; a < 3; ++a) H[(size_t)(3 * i + a) * n + 3 * i + a] += m.mass[i] * m.inv_dt2;
        for (int k = m.spr_off[i]; k < m.spr_off[i + 1]; ++k)
            for (int a = 0; a < 3; ++a) H[(size_t)(3 * i + a) * n + 3 * i + a] += m.spr_k[m.spr_list[k]];
        if (m.has_plane) {
            double sd = m.pn[0] * xi[0] + m.pn[1] * xi[1] + m.pn[2] * xi[2] - m.pd;
            if (sd < 0.0)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        H[(size_t)(3 * i + a) * n + 3 * i + b] += m.kc * m.pn[a] * m.pn[b];
        }
    }
}

// Chebyshev weights of Section "Acceleration Techniques": omega_{l+1} = 1 for
// l < 2, 2/(2 - rho^2) for l = 2 and 4/(4 - rho^2 omega_l) for l > 2.
double cheby_omega(int l, double omega_l, double rho) {
    if (l < 2) return 1.0;
    if (l == 2) return 2.0 / (2.0 - rho * rho);
    return 4.0 / (4.0 - rho * rho * omega_l);
}

}  // namespace

// ======================================================================== API
extern "C" {

void ora_lame(double E, double nu, double* mu, double* lam) {
    *mu = E / (2.0 * (1.0 + nu));
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

int ora_svd3(const double* F, double* U, double* s, double* V) { return svd3(F, U, s, V); }
void ora_polar(const double* F, double* R, double* shat) { polar(F, R, shat); }
double ora_psi(const double* F, double mu, double lam, int model) { return psi(F, mu, lam, model); }
void ora_pk1(const double* F, double mu, double lam, int model, double* P) { pk1(F, mu, lam, model, P); }
void ora_dpk1(const double* F, const double* dF, double mu, double lam, int model, double* dP) {
    dpk1(F, dF, mu, lam, model, dP);
}
void ora_cofactor(const double* F, double* C) { cof3(F, C); }

void ora_modified_density_hessian(const double* F, double mu, double lam, double* C81) {
    double C[9];
    cof3(F, C);
    for (int a = 0; a < 3; ++a)
        for (int g = 0; g < 3; ++g)
            for (int b = 0; b < 3; ++b)
                for (int d = 0; d < 3; ++d)
                    C81[(3 * a + g) * 9 + 3 * b + d] =
                        2.0 * mu * (a == b) * (g == d) + lam * C[3 * a + g] * C[3 * b + d];
}

void* ora_create(int nv, const double* X, int ne, const int* tets, const double* young,
                 const double* poisson, const unsigned char* is_dir, const double* body_accel,
                 const double* density, int ns, const int* spr_idx, const double* spr_t,
                 const double* spr_k, const double* plane, double k_contact, int* status) {
    *status = 1;
    if (nv <= 0 || ne < 0 || !X || (ne > 0 && !tets) || !young || !poisson) return nullptr;
    Mesh* m = new Mesh();
    m->nv = nv;
    m->ne = ne;
    m->X.assign(X, X + 3 * (size_t)nv);
    m->tets.assign(tets, tets + 4 * (size_t)ne);
    for (int v : m->tets)
        if (v < 0 || v >= nv) { delete m; return nullptr; }
    m->dir.assign(nv, 0);
    if (is_dir)
        for (int i = 0; i < nv; ++i) m->dir[i] = is_dir[i] ? 1 : 0;
    m->mu.resize(ne);
    m->lam.resize(ne);
    m->vol.resize(ne);
    m->B.resize(9 * (size_t)ne);
    for (int e = 0; e < ne; ++e) {
        // Dm = [X1-X0, X2-X0, X3-X0] (columns); B = Dm^{-1}; V^0 = |det Dm|/6.
        const int* t = &m->tets[4 * (size_t)e];
        double Dm[9], C[9];
        double hmax = 0.0;
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 3; ++a) {
                Dm[3 * a + c] = X[3 * (size_t)t[c + 1] + a] - X[3 * (size_t)t[0] + a];
                hmax = std::max(hmax, std::fabs(Dm[3 * a + c]));
            }
        double D = det3(Dm);
        if (!(std::fabs(D) / 6.0 > 1e-12 * hmax * hmax * hmax)) { delete m; *status = 4; return nullptr; }
        cof3(Dm, C);  // Dm^{-1} = cof(Dm)^T / det
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) m->B[9 * (size_t)e + 3 * a + b] = C[3 * b + a] / D;
        m->vol[e] = std::fabs(D) / 6.0;
        ora_lame(young[e], poisson[e], &m->mu[e], &m->lam[e]);
    }
    // Vertex -> incident (tet, local index), ascending tet id.
    m->inc_off.assign(nv + 1, 0);
    for (int v : m->tets) m->inc_off[v + 1]++;
    for (int i = 0; i < nv; ++i) m->inc_off[i + 1] += m->inc_off[i];
    m->inc_tet.resize(4 * (size_t)ne);
    m->inc_loc.resize(4 * (size_t)ne);
    std::vector<int> fill(m->inc_off.begin(), m->inc_off.end() - 1);
    for (int e = 0; e < ne; ++e)
        for (int j = 0; j < 4; ++j) {
            int v = m->tets[4 * (size_t)e + j];
            m->inc_tet[fill[v]] = e;
            m->inc_loc[fill[v]] = j;
            fill[v]++;
        }
    // f^ext_i = int f N_i dX = rho_e a V_e / 4 per incident tet for a constant
    // body acceleration a (P1 shape functions integrate to V/4).
    m->fext.assign(3 * (size_t)nv, 0.0);
    if (body_accel && density)
        for (int e = 0; e < ne; ++e)
            for (int j = 0; j < 4; ++j)
                for (int a = 0; a < 3; ++a)
                    m->fext[3 * (size_t)m->tets[4 * (size_t)e + j] + a] +=
                        density[e] * body_accel[a] * m->vol[e] / 4.0;
    m->spr_off.assign(nv + 1, 0);
    for (int s = 0; s < ns; ++s) {
        if (spr_idx[s] < 0 || spr_idx[s] >= nv) { delete m; return nullptr; }
        m->spr_off[spr_idx[s] + 1]++;
    }
    for (int i = 0; i < nv; ++i) m->spr_off[i + 1] += m->spr_off[i];
    m->spr_list.resize(ns);
    std::vector<int> sf(m->spr_off.begin(), m->spr_off.end() - 1);
    for (int s = 0; s < ns; ++s) m->spr_list[sf[spr_idx[s]]++] = s;
    if (ns > 0) {
        m->spr_t.assign(spr_t, spr_t + 3 * (size_t)ns);
        m->spr_k.assign(spr_k, spr_k + ns);
    }
    if (plane) {
        m->has_plane = true;
        for (int a = 0; a < 3; ++a) m->pn[a] = plane[a];
        m->pd = plane[3];
        m->kc = k_contact;
    }
    m->vert_wc.assign(nv, {});
    colour_nodes(*m);
    *status = 0;
    return m;
}

void ora_destroy(void* h) { delete static_cast<Mesh*>(h); }

// Backward Euler of Eq. fem_be with the lumped mass m_ii = sum_e rho_e V_e / 4
// (the integral of R^0 N_i for P1 tets).  dt <= 0 returns to quasistatics.
int ora_set_inertia(void* h, double dt, const double* density, const double* xhat) {
    Mesh& m = *static_cast<Mesh*>(h);
    if (!(dt > 0.0)) {
        m.inv_dt2 = 0.0;
        return 0;
    }
    if (!density || !xhat) return 1;
    m.mass.assign(m.nv, 0.0);
    for (int e = 0; e < m.ne; ++e)
        for (int j = 0; j < 4; ++j) m.mass[m.tets[4 * (size_t)e + j]] += density[e] * m.vol[e] / 4.0;
    m.xhat.assign(xhat, xhat + 3 * (size_t)m.nv);
    m.inv_dt2 = 1.0 / (dt * dt);
    return 0;
}

void ora_lumped_mass(const void* h, double* out) {
    const Mesh& m = *static_cast<const Mesh*>(h);
    for (int i = 0; i < m.nv; ++i) out[i] = m.mass.empty() ? 0.0 : m.mass[i];
}

// General weak constraints (Section "Weak Constraints").  Constraint c has
// up to 4 nodes per side: idx[8c + k] (-1 = unused), weights w[8c + k] >= 0
// with k < 4 on side 0 and k >= 4 on side 1, each used side summing to one;
// stiffness K_c = kt I + (kn - kt) n n^T with |n| = 1.  recolour = 0 colours
// every node again greedily; 1 keeps the current colours and revisits the
// constraint nodes (Section "Collision Coloring").  Returns nonzero on bad
// input.
int ora_set_weak_constraints(void* h, int nc, const int* idx, const double* w, const double* kn, const double* kt,
                             const double* nrm, int recolour) {
    Mesh& m = *static_cast<Mesh*>(h);
    std::vector<std::vector<int>> cv(nc);
    std::vector<std::vector<double>> cb(nc);
    std::vector<std::array<double, 9>> cK(nc);
    for (int c = 0; c < nc; ++c) {
        double sum[2] = {0.0, 0.0};
        for (int k = 0; k < 8; ++k) {
            const int v = idx[8 * c + k];
            const double wk = w[8 * c + k];
            if (v < 0) continue;
            if (v >= m.nv || !(wk >= 0.0)) return 1;
            sum[k / 4] += wk;
            const double coef = k < 4 ? wk : -wk;
            size_t p = 0;
            while (p < cv[c].size() && cv[c][p] != v) ++p;
            if (p == cv[c].size()) {
                cv[c].push_back(v);
                cb[c].push_back(coef);
            } else {
                cb[c][p] += coef;
            }
        }
        if (std::fabs(sum[0] - 1.0) > 1e-9 || std::fabs(sum[1] - 1.0) > 1e-9) return 1;
        const double* n = &nrm[3 * c];
        const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0.0) || !(kn[c] >= 0.0) || !(kt[c] >= 0.0)) return 1;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                cK[c][3 * a + b] = (a == b ? kt[c] : 0.0) + (kn[c] - kt[c]) * n[a] * n[b] / (nn * nn);
    }
    m.wc_v = std::move(cv);
    m.wc_b = std::move(cb);
    m.wc_K = std::move(cK);
    m.vert_wc.assign(m.nv, {});
    for (int c = 0; c < nc; ++c)
        for (int v : m.wc_v[c]) m.vert_wc[v].push_back(c);
    if (recolour) recolour_constraint_nodes(m);
    else colour_nodes(m);
    return 0;
}

int ora_set_model(void* h, int model) {
    if (model < kCorotated || model > kStableNeoHookean) return 1;
    static_cast<Mesh*>(h)->model = model;
    return 0;
}

int ora_set_colour_order(void* h, int order) {
    if (order != 0 && order != 1) return 1;
    static_cast<Mesh*>(h)->colour_order = order;
    return 0;
}

int ora_num_colours(const void* h) { return (int)static_cast<const Mesh*>(h)->by_colour.size(); }

void ora_get_colours(const void* h, int* colour) {
    const Mesh* m = static_cast<const Mesh*>(h);
    std::copy(m->colour.begin(), m->colour.end(), colour);
}

void ora_get_tet_constants(const void* h, double* B9, double* V, double* mu, double* lam) {
    const Mesh* m = static_cast<const Mesh*>(h);
    if (B9) std::copy(m->B.begin(), m->B.end(), B9);
    if (V) std::copy(m->vol.begin(), m->vol.end(), V);
    if (mu) std::copy(m->mu.begin(), m->mu.end(), mu);
    if (lam) std::copy(m->lam.begin(), m->lam.end(), lam);
}

void ora_get_fext(const void* h, double* f) {
    const Mesh* m = static_cast<const Mesh*>(h);
    std::copy(m->fext.begin(), m->fext.end(), f);
}

void ora_local_system(const void* h, const double* x, int i, double* r3, double* A9) {
    local_system(*static_cast<const Mesh*>(h), x, i, r3, A9);
}

double ora_residual(const void* h, const double* x, double* r_out) {
    return residual(*static_cast<const Mesh*>(h), x, r_out);
}

double ora_energy(const void* h, const double* x) { return energy(*static_cast<const Mesh*>(h), x); }

int ora_sweeps(const void* h, double* x, int nsweeps, int accel, double omega, double rho,
               double gamma, double skip_tol, int nthreads, double* res_hist) {
    const Mesh& m = *static_cast<const Mesh*>(h);
    const size_t n3 = 3 * (size_t)m.nv;
    std::vector<double> x_prev(x, x + n3), x_prev2(x, x + n3);  // x^l, x^{l-1}
    if (res_hist) res_hist[0] = residual(m, x, nullptr);
    double om = 1.0;
    int bad = 0;
    for (int l = 0; l < nsweeps; ++l) {
        // One PBNG iteration: colours in ascending order (Section "Coloring
        // and Parallelism"); nodes of one colour share no element, so their
        // order inside the colour does not change the result.
        // With the symmetric order the sweep goes back down after the last
        // colour (0..C-1, C-2..0), the palindromic colour sequence of a
        // symmetric Gauss-Seidel iteration.
        const int C = (int)m.by_colour.size();
        const int npass = (m.colour_order == 1 && C > 0) ? 2 * C - 1 : C;
        for (int t = 0; t < npass; ++t) {
            const auto& list = m.by_colour[t < C ? t : 2 * C - 2 - t];
            const int cnt = (int)list.size();
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : bad)
            for (int q = 0; q < cnt; ++q)
                if (!node_update(m, x, list[q], skip_tol)) bad += 1;
        }
        if (accel == 1 || accel == 2) {
            // Chebyshev: x^{l+1} = w_{l+1}(g(x_P - x^l) + x^l - x^{l-1}) + x^{l-1};
            // SOR as printed: x^{l+1} = w(x_P - x^{l-1}) + x^{l-1}.
            double w, g;
            if (accel == 1) { om = cheby_omega(l, om, rho); w = om; g = gamma; }
            else { w = omega; g = 1.0; }
            for (int i = 0; i < m.nv; ++i) {
                if (m.dir[i]) continue;
                for (int a = 0; a < 3; ++a) {
                    size_t k = 3 * (size_t)i + a;
                    double xp = x[k];
                    double xn = w * (g * (xp - x_prev[k]) + x_prev[k] - x_prev2[k]) + x_prev2[k];
                    x_prev2[k] = x_prev[k];
                    x_prev[k] = xn;
                    x[k] = xn;
                }
            }
        }
        if (res_hist) res_hist[l + 1] = residual(m, x, nullptr);
    }
    return bad ? 5 : 0;
}

int ora_newton(const void* h, double* x, double rel_tol, int maxit, double* res_out) {
    const Mesh& m = *static_cast<const Mesh*>(h);
    const int n = 3 * m.nv;
    std::vector<int> fdof;
    for (int i = 0; i < m.nv; ++i)
        if (!m.dir[i])
            for (int a = 0; a < 3; ++a) fdof.push_back(3 * i + a);
    const int nf = (int)fdof.size();
    std::vector<double> r(n), H, Hf, b;
    double r0 = residual(m, x, r.data()), rn = r0;
    int it = 0;
    for (; it < maxit && rn > rel_tol * r0; ++it) {
        hessian_dense(m, x, H);
        Hf.assign((size_t)nf * nf, 0.0);
        b.assign(nf, 0.0);
        for (int p = 0; p < nf; ++p) {
            b[p] = r[fdof[p]];
            for (int q = 0; q < nf; ++q) Hf[(size_t)p * nf + q] = H[(size_t)fdof[p] * n + fdof[q]];
        }
        std::vector<double> d = b;
        double shift = 0.0;
        // Levenberg shift until the step is a descent direction (H may be indefinite).
        for (int tries = 0; tries < 30; ++tries) {
            std::vector<double> A = Hf;
            for (int p = 0; p < nf; ++p) A[(size_t)p * nf + p] += shift;
            d = b;
            bool ok = lu_solve(A, d, nf);
            double dot = 0.0;
            for (int p = 0; p < nf; ++p) dot += d[p] * b[p];
            if (ok && dot > 0.0) break;
            double diag = 0.0;
            for (int p = 0; p < nf; ++p) diag = std::max(diag, std::fabs(Hf[(size_t)p * nf + p]));
            shift = (shift == 0.0) ? 1e-6 * diag : 10.0 * shift;
        }
        // Backtracking on the energy.  Near the solution the predicted energy
        // decrease alpha (d . r) falls below the rounding of E itself; there a
        // step that lowers the residual norm is accepted instead.
        double E0 = energy(m, x), alpha = 1.0, dr = 0.0;
        for (int p = 0; p < nf; ++p) dr += d[p] * b[p];
        std::vector<double> xt(x, x + n);
        for (int ls = 0; ls < 40; ++ls) {
            for (int p = 0; p < nf; ++p) xt[fdof[p]] = x[fdof[p]] + alpha * d[p];
            if (energy(m, xt.data()) <= E0) break;
            if (alpha * dr < 1e-12 * std::fabs(E0) && residual(m, xt.data(), nullptr) < rn) break;
            alpha *= 0.5;
        }
        std::copy(xt.begin(), xt.end(), x);
        rn = residual(m, x, r.data());
    }
    if (res_out) *res_out = rn / (r0 > 0 ? r0 : 1.0);
    return (rn <= rel_tol * r0) ? it : -1;
}

void ora_hessian_dense(const void* h, const double* x, double* Hout) {
    const Mesh& m = *static_cast<const Mesh*>(h);
    std::vector<double> H;
    hessian_dense(m, x, H);
    std::copy(H.begin(), H.end(), Hout);
}

int ora_adjoint_dense(const void* h, const double* x, const double* dLdx, double* dLdlogE,
                      double* dLdxD) {
    const Mesh& m = *static_cast<const Mesh*>(h);
    const int n = 3 * m.nv;
    std::vector<double> H;
    hessian_dense(m, x, H);
    std::vector<int> fdof, ddof;
    for (int i = 0; i < m.nv; ++i)
        for (int a = 0; a < 3; ++a) (m.dir[i] ? ddof : fdof).push_back(3 * i + a);
    const int nf = (int)fdof.size();
    std::vector<double> Hf((size_t)nf * nf), lamv(nf);
    for (int p = 0; p < nf; ++p) {
        lamv[p] = dLdx[fdof[p]];
        for (int q = 0; q < nf; ++q) Hf[(size_t)p * nf + q] = H[(size_t)fdof[p] * n + fdof[q]];
    }
    if (!lu_solve(Hf, lamv, nf)) return 1;
    std::vector<double> lam_full(n, 0.0);
    for (int p = 0; p < nf; ++p) lam_full[fdof[p]] = lamv[p];
    // d r_i / d log E_e = -V_e P_e g_i (P is linear in (mu, lambda), both ~ E).
    for (int e = 0; e < m.ne; ++e) {
        double F[9], P[9], s = 0.0;
        deformation_gradient(m, x, e, F);
        pk1(F, m.mu[e], m.lam[e], m.model, P);
        for (int j = 0; j < 4; ++j) {
            int v = m.tets[4 * (size_t)e + j];
            if (m.dir[v]) continue;
            double g[3], Pg[3];
            grad(m, e, j, g);
            mat_vec(P, g, Pg);
            for (int a = 0; a < 3; ++a) s -= lam_full[3 * (size_t)v + a] * m.vol[e] * Pg[a];
        }
        dLdlogE[e] = s;
    }
    for (size_t p = 0; p < ddof.size(); ++p) {
        double s = dLdx[ddof[p]];
        for (int q = 0; q < nf; ++q) s -= H[(size_t)ddof[p] * n + fdof[q]] * lamv[q];
        dLdxD[p] = s;
    }
    return 0;
}

int ora_threads_available(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? std::min(nthreads, omp_get_num_procs()) : 1;
#else
    (void)nthreads;
    return 1;
#endif
}

}  // extern "C"
