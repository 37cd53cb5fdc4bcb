// setup.cpp -- host-side (FP64) construction of the MGMC hierarchy (Sec. 2.3-2.5).
//
//  - finest operator A_L = s (kappa^2 I - Delta_h), s = h^d or 1, its Q1
//    finite-element matrix, or the 13-point matrix of the squared shifted
//    Laplacian s (kappa^2 - Delta_h)^2 with u = du/dn = 0 (2D; Sec. 5.1.1), whose
//    grids all carry radius-2 (5 x 5) stencils;
//  - Galerkin coarse operators A_{l-1} = P^T A_l P (Eq. A_ell_1_B_ell_1): entry
//    (J, J+q) = (P e_J)^T A (P e_{J+q}), the product of the two coarse hat
//    functions through A, summed over the fine sites where both are nonzero;
//  - B_{l-1} = P^T B_l;
//  - per level and direction the low-rank matrices of Alg. 3:
//    C = M^-1 B (M = D + L or D + L^T in colour order), S = Gamma + B^T C,
//    G = C S^-1.  Each column of C is a forward substitution started from
//    zero; a colour pass can only extend the support by one stencil radius,
//    so the substitution runs on the bounding box of supp(b_k) grown by the
//    radius times (the number of colours + 1), which gives the full-grid result;
//  - the coarsest posterior operator A~_0 = A_0 + B_0 Gamma^-1 B_0^T and its
//    Cholesky factor (exact coarse sampler, Sec. 3.5);
//  - the finest data vector d_L = y, so that f_L = B_L Gamma^-1 d_L (Eq. f_ell_definition).
#include "setup.hpp"

#include <algorithm>
#include <cmath>
#include <map>

#include "../../include/mgmc.h"

namespace mgmc {

namespace {

struct Grid {
    int d, n;
    long long idx(int i, int j, int k) const { return i + (long long)n * (j + (long long)n * k); }
    bool inside(int i, int j, int k) const
    {
        return i >= 0 && i < n && j >= 0 && j < n && (d == 2 ? k == 0 : (k >= 0 && k < n));
    }
    void coords(long long s, int& i, int& j, int& k) const
    {
        i = (int)(s % n);
        j = (int)((s / n) % n);
        k = d == 3 ? (int)(s / ((long long)n * n)) : 0;
    }
};

// offset index of (dx, dy, dz) in a full stencil of radius R: width W = 2R + 1, dx fastest
inline int oidx(int d, int R, int dx, int dy, int dz)
{
    const int W = 2 * R + 1;
    return (dx + R) + W * (dy + R) + (d == 3 ? W * W * (dz + R) : 0);
}

// hat function of coarse vertex J (1D) at fine vertex i: 1 at i = 2J+1, 1/2 at 2J, 2J+2
inline double hat(int J, int i)
{
    int t = i - (2 * J + 1);
    return t == 0 ? 1.0 : (t == 1 || t == -1) ? 0.5 : 0.0;
}

// colour order of the Gibbs sweep: parity classes (radius 1); radius-2 stencils (2D)
// the nine classes (i mod 3, j mod 3), code (i mod 3) + 3 (j mod 3), in code order
std::vector<int> colour_order(int d, int R)
{
    if (R == 2) return {0, 1, 2, 3, 4, 5, 6, 7, 8};
    if (d == 2) return {0, 3, 2, 1};
    return {0, 6, 5, 3, 4, 2, 1, 7};
}

int colour_of(int d, int R, int i, int j, int k)
{
    if (R == 2) return i % 3 + 3 * (j % 3);
    return (i & 1) | ((j & 1) << 1) | (d == 3 ? ((k & 1) << 2) : 0);
}

bool lu_inverse(int k, std::vector<double> A, std::vector<double>& inv)
{
    inv.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) inv[(size_t)i * k + i] = 1.0;
    for (int c = 0; c < k; ++c) {
        int p = c;
        for (int r = c + 1; r < k; ++r)
            if (std::fabs(A[(size_t)r * k + c]) > std::fabs(A[(size_t)p * k + c])) p = r;
        if (A[(size_t)p * k + c] == 0.0 || !std::isfinite(A[(size_t)p * k + c])) return false;
        if (p != c)
            for (int t = 0; t < k; ++t) {
                std::swap(A[(size_t)p * k + t], A[(size_t)c * k + t]);
                std::swap(inv[(size_t)p * k + t], inv[(size_t)c * k + t]);
            }
        double piv = A[(size_t)c * k + c];
        for (int r = 0; r < k; ++r) {
            if (r == c) continue;
            double f = A[(size_t)r * k + c] / piv;
            if (f == 0.0) continue;
            for (int t = 0; t < k; ++t) {
                A[(size_t)r * k + t] -= f * A[(size_t)c * k + t];
                inv[(size_t)r * k + t] -= f * inv[(size_t)c * k + t];
            }
        }
    }
    for (int r = 0; r < k; ++r) {
        double piv = A[(size_t)r * k + r];
        for (int t = 0; t < k; ++t) inv[(size_t)r * k + t] /= piv;
    }
    return true;
}

bool cholesky_lower(int k, const std::vector<double>& A, std::vector<double>& L)
{
    L.assign((size_t)k * k, 0.0);
    for (int c = 0; c < k; ++c) {
        double dsum = A[(size_t)c * k + c];
        for (int t = 0; t < c; ++t) dsum -= L[(size_t)c * k + t] * L[(size_t)c * k + t];
        if (!(dsum > 0.0) || !std::isfinite(dsum)) return false;
        double lcc = std::sqrt(dsum);
        L[(size_t)c * k + c] = lcc;
        for (int r = c + 1; r < k; ++r) {
            double v = A[(size_t)r * k + c];
            for (int t = 0; t < c; ++t) v -= L[(size_t)r * k + t] * L[(size_t)c * k + t];
            L[(size_t)r * k + c] = v / lcc;
        }
    }
    return true;
}

void galerkin(const HostProblem& hp, const HostLevel& F, HostLevel& Cl)
{
    const int d = hp.dim, NS = hp.NS, R = hp.R;
    Grid gf{d, F.n}, gc{d, Cl.n};
    Cl.st.assign((size_t)Cl.N * NS, 0.0);
    const int kz = d == 3 ? 1 : 0, rz = d == 3 ? R : 0;
    for (long long J = 0; J < Cl.N; ++J) {
        int I0, I1, I2;
        gc.coords(J, I0, I1, I2);
        double* out = &Cl.st[(size_t)J * NS];
        // fine sites in the patch of J
        for (int pz = -kz; pz <= kz; ++pz)
            for (int py = -1; py <= 1; ++py)
                for (int px = -1; px <= 1; ++px) {
                    int fi = 2 * I0 + 1 + px, fj = 2 * I1 + 1 + py, fk = d == 3 ? 2 * I2 + 1 + pz : 0;
                    double wJ = hat(I0, fi) * hat(I1, fj) * (d == 3 ? hat(I2, fk) : 1.0);
                    const double* a = &F.st[(size_t)gf.idx(fi, fj, fk) * NS];
                    for (int oz = -rz; oz <= rz; ++oz)
                        for (int oy = -R; oy <= R; ++oy)
                            for (int ox = -R; ox <= R; ++ox) {
                                double aij = a[oidx(d, R, ox, oy, oz)];
                                if (aij == 0.0) continue;
                                int gi = fi + ox, gj = fj + oy, gk = fk + oz;
                                if (!gf.inside(gi, gj, gk)) continue;
                                // coarse neighbours K = J + q whose hat covers (gi, gj, gk)
                                for (int qz = -rz; qz <= rz; ++qz)
                                    for (int qy = -R; qy <= R; ++qy)
                                        for (int qx = -R; qx <= R; ++qx) {
                                            int K0 = I0 + qx, K1 = I1 + qy, K2 = I2 + qz;
                                            if (!gc.inside(K0, K1, K2)) continue;
                                            double wK = hat(K0, gi) * hat(K1, gj) * (d == 3 ? hat(K2, gk) : 1.0);
                                            if (wK == 0.0) continue;
                                            out[oidx(d, R, qx, qy, qz)] += wJ * aij * wK;
                                        }
                            }
                }
    }
}

void coarsen_B(const HostProblem& hp, const HostLevel& F, HostLevel& Cl)
{
    const int d = hp.dim;
    Grid gf{d, F.n}, gc{d, Cl.n};
    Cl.bptr.assign(hp.m + 1, 0);
    Cl.bsite.clear();
    Cl.bw.clear();
    for (int k = 0; k < hp.m; ++k) {
        std::map<long long, double> col;
        for (int t = F.bptr[k]; t < F.bptr[k + 1]; ++t) {
            int i, j, kk;
            gf.coords(F.bsite[t], i, j, kk);
            // coarse vertices with i in their hat support: floor((i-1)/2) .. ceil((i-1)/2)
            for (int c2 = (d == 3 ? (kk - 2) / 2 : 0); c2 <= (d == 3 ? kk / 2 : 0); ++c2)
                for (int c1 = (j - 2) / 2; c1 <= j / 2; ++c1)
                    for (int c0 = (i - 2) / 2; c0 <= i / 2; ++c0) {
                        if (!gc.inside(c0, c1, c2)) continue;
                        double w = hat(c0, i) * hat(c1, j) * (d == 3 ? hat(c2, kk) : 1.0);
                        if (w != 0.0) col[gc.idx(c0, c1, c2)] += w * F.bw[t];
                    }
        }
        for (auto& kv : col)
            if (kv.second != 0.0) {
                Cl.bsite.push_back(kv.first);
                Cl.bw.push_back(kv.second);
            }
        Cl.bptr[k + 1] = (int)Cl.bsite.size();
    }
}

// C_k = M^-1 b_k on a box; returns the nonzero (site, value) pairs
void lower_solve_column(const HostProblem& hp, const HostLevel& L, int dir, int k,
                        std::vector<std::pair<long long, double>>& out)
{
    const int d = hp.dim, NS = hp.NS, n = L.n, R = hp.R;
    Grid g{d, n};
    std::vector<int> order = colour_order(d, R);
    if (dir == 1) std::reverse(order.begin(), order.end());
    int lo[3] = {n, n, n}, hi[3] = {-1, -1, -1};
    std::map<long long, double> b;
    for (int t = L.bptr[k]; t < L.bptr[k + 1]; ++t) {
        int c[3];
        g.coords(L.bsite[t], c[0], c[1], c[2]);
        for (int a = 0; a < d; ++a) {
            lo[a] = std::min(lo[a], c[a]);
            hi[a] = std::max(hi[a], c[a]);
        }
        b[L.bsite[t]] += L.bw[t];
    }
    out.clear();
    if (b.empty()) return;
    const int grow = R * ((int)order.size() + 1);
    int blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) {
        blo[a] = std::max(0, lo[a] - grow);
        bhi[a] = std::min(n - 1, hi[a] + grow);
        ext[a] = bhi[a] - blo[a] + 1;
    }
    std::vector<double> box((size_t)ext[0] * ext[1] * ext[2], 0.0);
    auto bidx = [&](int i, int j, int kk) {
        return (size_t)(i - blo[0]) + (size_t)ext[0] * ((j - blo[1]) + (size_t)ext[1] * (kk - blo[2]));
    };
    const int rz = d == 3 ? R : 0;
    for (int colour : order) {
        for (int kk = blo[2]; kk <= bhi[2]; ++kk)
            for (int j = blo[1]; j <= bhi[1]; ++j)
                for (int i = blo[0]; i <= bhi[0]; ++i) {
                    if (colour_of(d, R, i, j, kk) != colour) continue;
                    long long s = g.idx(i, j, kk);
                    const double* a = &L.st[(size_t)s * NS];
                    auto it = b.find(s);
                    double acc = it == b.end() ? 0.0 : it->second;
                    for (int oz = -rz; oz <= rz; ++oz)
                        for (int oy = -R; oy <= R; ++oy)
                            for (int ox = -R; ox <= R; ++ox) {
                                if (ox == 0 && oy == 0 && oz == 0) continue;
                                double aij = a[oidx(d, R, ox, oy, oz)];
                                if (aij == 0.0) continue;
                                int i2 = i + ox, j2 = j + oy, k2 = kk + oz;
                                if (i2 < blo[0] || i2 > bhi[0] || j2 < blo[1] || j2 > bhi[1] || k2 < blo[2] ||
                                    k2 > bhi[2])
                                    continue;   // outside the box the column is still zero
                                acc -= aij * box[bidx(i2, j2, k2)];
                            }
                    box[bidx(i, j, kk)] = acc / a[hp.C];
                }
    }
    for (int kk = blo[2]; kk <= bhi[2]; ++kk)
        for (int j = blo[1]; j <= bhi[1]; ++j)
            for (int i = blo[0]; i <= bhi[0]; ++i) {
                double v = box[bidx(i, j, kk)];
                if (v != 0.0) out.emplace_back(g.idx(i, j, kk), v);
            }
}

bool lowrank_setup(const HostProblem& hp, HostLevel& L, int dir)
{
    const int m = hp.m;
    L.gsite[dir].clear();
    L.gval[dir].clear();
    if (m == 0) return true;
    std::map<long long, std::vector<double>> Crows;   // support site -> row of C
    std::vector<std::pair<long long, double>> col;
    for (int k = 0; k < m; ++k) {
        lower_solve_column(hp, L, dir, k, col);
        for (auto& e : col) {
            auto& row = Crows[e.first];
            if (row.empty()) row.assign(m, 0.0);
            row[k] = e.second;
        }
    }
    // S = Gamma + B^T C
    std::vector<double> S(hp.Gamma);
    for (int k = 0; k < m; ++k)
        for (int t = L.bptr[k]; t < L.bptr[k + 1]; ++t) {
            auto it = Crows.find(L.bsite[t]);
            if (it == Crows.end()) continue;
            for (int j = 0; j < m; ++j) S[(size_t)k * m + j] += L.bw[t] * it->second[j];
        }
    std::vector<double> Sinv;
    if (!lu_inverse(m, S, Sinv)) return false;
    for (auto& kv : Crows) {
        L.gsite[dir].push_back(kv.first);
        for (int j = 0; j < m; ++j) {
            double acc = 0.0;
            for (int k = 0; k < m; ++k) acc += kv.second[k] * Sinv[(size_t)k * m + j];
            L.gval[dir].push_back(acc);
        }
    }
    return true;
}

}  // namespace

void fused_extras(HostLevel& L, const HostProblem& hp, int l)
{
    const HostLevel& Cl = hp.lev[l - 1];
    const int d = hp.dim, m = hp.m, R = hp.R, rz = d == 3 ? R : 0;
    L.hsite.clear();
    L.hval.clear();
    L.BtG.assign((size_t)m * m, 0.0);
    if (m == 0) return;
    Grid g{d, L.n}, gc{d, Cl.n};
    // A G on the fine grid: column-wise (A G)_j = sum_s a_{j s} G_s, a symmetric
    std::map<long long, std::vector<double>> AG;
    std::map<long long, size_t> grow;
    for (size_t r = 0; r < L.gsite[0].size(); ++r) {
        long long s = L.gsite[0][r];
        grow[s] = r;
        int i, j, k;
        g.coords(s, i, j, k);
        const double* a = &L.st[(size_t)s * hp.NS];
        for (int oz = -rz; oz <= rz; ++oz)
            for (int oy = -R; oy <= R; ++oy)
                for (int ox = -R; ox <= R; ++ox) {
                    double aso = a[oidx(d, R, ox, oy, oz)];
                    if (aso == 0.0 || !g.inside(i + ox, j + oy, k + oz)) continue;
                    auto& v = AG[g.idx(i + ox, j + oy, k + oz)];
                    if (v.empty()) v.assign(m, 0.0);
                    for (int c = 0; c < m; ++c) v[c] += aso * L.gval[0][r * m + c];
                }
    }
    // H = P^T (A G)
    std::map<long long, std::vector<double>> H;
    for (auto& kv : AG) {
        int i, j, k;
        g.coords(kv.first, i, j, k);
        for (int c2 = (d == 3 ? (k - 2) / 2 : 0); c2 <= (d == 3 ? k / 2 : 0); ++c2)
            for (int c1 = (j - 2) / 2; c1 <= j / 2; ++c1)
                for (int c0 = (i - 2) / 2; c0 <= i / 2; ++c0) {
                    if (!gc.inside(c0, c1, c2)) continue;
                    double w = hat(c0, i) * hat(c1, j) * (d == 3 ? hat(c2, k) : 1.0);
                    if (w == 0.0) continue;
                    auto& v = H[gc.idx(c0, c1, c2)];
                    if (v.empty()) v.assign(m, 0.0);
                    for (int c = 0; c < m; ++c) v[c] += w * kv.second[c];
                }
    }
    for (auto& kv : H) {
        L.hsite.push_back(kv.first);
        L.hval.insert(L.hval.end(), kv.second.begin(), kv.second.end());
    }
    // B^T G
    for (int k = 0; k < m; ++k)
        for (int t = L.bptr[k]; t < L.bptr[k + 1]; ++t) {
            auto it = grow.find(L.bsite[t]);
            if (it == grow.end()) continue;
            for (int c = 0; c < m; ++c) L.BtG[(size_t)k * m + c] += L.bw[t] * L.gval[0][it->second * m + c];
        }
}

std::vector<double> row_sums(const HostProblem& hp, int l)
{
    const HostLevel& L = hp.lev[l];
    Grid g{hp.dim, L.n};
    std::vector<double> out((size_t)L.N, 0.0);
    const int R = hp.R, rz = hp.dim == 3 ? R : 0;
    for (long long s = 0; s < L.N; ++s) {
        int i, j, k;
        g.coords(s, i, j, k);
        double acc = 0.0;
        for (int oz = -rz; oz <= rz; ++oz)
            for (int oy = -R; oy <= R; ++oy)
                for (int ox = -R; ox <= R; ++ox)
                    if (g.inside(i + ox, j + oy, k + oz))
                        acc += L.st[(size_t)s * hp.NS + oidx(hp.dim, R, ox, oy, oz)];
        out[(size_t)s] = acc;
    }
    return out;
}

// The finest grid's operator into hp.lev[top].st (and, finite differences, the
// s kappa^2 part and s / h^2 of the FP32 form); empty string on success.
std::string fine_operator(HostProblem& hp, int dim, int n, int scale_hd, int disc, const double* kappa2,
                          double kappa2_const)
{
    HostLevel& Fl = hp.lev[hp.n_levels - 1];
    Grid gf{dim, n};
    const double h = 1.0 / (double)(n + 1);
    double scale = 1.0;
    if (scale_hd)
        for (int a = 0; a < dim; ++a) scale *= h;
    const double inv_h2 = 1.0 / (h * h);
    hp.woff_fine = scale * inv_h2;
    Fl.st.assign((size_t)Fl.N * hp.NS, 0.0);
    hp.kappa_part.assign((size_t)Fl.N, 0.0);
    // Q1 elements: per offset o the 1D integrals of hat functions, one derivative pair per
    // axis -- stiffness (2, -1) / h, mass (4, 1) h / 6 for |o_t| = 0, 1 -- multiplied out
    std::vector<double> q1(hp.NS, 0.0);
    if (disc == 1) {
        if (!std::isfinite(kappa2_const) || kappa2_const < 0.0) return "kappa^2 must be finite and non-negative";
        double hd = 1.0;
        for (int a = 0; a < dim; ++a) hd *= h;
        const double q1scale = scale_hd ? 1.0 : 1.0 / hd;   // literal scaling: the FE matrix divided by h^d
        for (int o = 0; o < hp.NS; ++o) {
            const int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
            double stiff = 0.0, mass = 1.0;
            for (int ax = 0; ax < dim; ++ax) {
                double tk = off[ax] == 0 ? 2.0 / h : -1.0 / h;
                for (int t = 0; t < dim; ++t)
                    if (t != ax) tk *= off[t] == 0 ? 4.0 * h / 6.0 : h / 6.0;
                stiff += tk;
                mass *= off[ax] == 0 ? 4.0 * h / 6.0 : h / 6.0;
            }
            q1[(size_t)o] = q1scale * (stiff + kappa2_const * mass);
        }
    }
    if (disc == 2) {
        // (kappa^2 - Delta_h)^2 with u = du/dn = 0 as the product K K of the shifted
        // 5-point Dirichlet operator K = kappa^2 + L (L = -Delta_h) with itself, plus
        // 2 h^-4 per boundary side a vertex is adjacent to: the 13-point stencil's
        // mirror ghost behind the boundary adds h^-4 to such a row, where K K misses
        // the h^-4 of the dropped boundary vertex (Sec. 5.1.1)
        if (!std::isfinite(kappa2_const) || kappa2_const < 0.0) return "kappa^2 must be finite and non-negative";
        const double kc = kappa2_const + 4.0 * inv_h2, ko = -inv_h2;
        const int nb[5][2] = {{0, 0}, {-1, 0}, {1, 0}, {0, -1}, {0, 1}};
        for (long long s = 0; s < Fl.N; ++s) {
            int i, j, k;
            gf.coords(s, i, j, k);
            double* a = &Fl.st[(size_t)s * hp.NS];
            for (int t = 0; t < 5; ++t) {
                const int ti = i + nb[t][0], tj = j + nb[t][1];
                if (!gf.inside(ti, tj, 0)) continue;
                const double kst = t == 0 ? kc : ko;
                for (int u = 0; u < 5; ++u) {
                    const int ui = ti + nb[u][0], uj = tj + nb[u][1];
                    if (!gf.inside(ui, uj, 0)) continue;
                    a[oidx(2, 2, ui - i, uj - j, 0)] += scale * kst * (u == 0 ? kc : ko);
                }
            }
            const int sides = (i == 0) + (i == n - 1) + (j == 0) + (j == n - 1);
            a[hp.C] += scale * 2.0 * inv_h2 * inv_h2 * sides;
        }
        return std::string();
    }
    for (long long s = 0; s < Fl.N; ++s) {
        double k2 = kappa2 ? kappa2[s] : kappa2_const;
        if (!std::isfinite(k2) || k2 < 0.0) return "kappa^2 must be finite and non-negative";
        int i, j, k;
        gf.coords(s, i, j, k);
        double* a = &Fl.st[(size_t)s * hp.NS];
        if (disc == 1) {
            for (int o = 0; o < hp.NS; ++o) {
                const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
                if (gf.inside(i + ox, j + oy, dim == 3 ? k + oz : k)) a[o] = q1[(size_t)o];
            }
            continue;
        }
        a[hp.C] = scale * (k2 + 2.0 * dim * inv_h2);
        hp.kappa_part[(size_t)s] = scale * k2;
        const int dd[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
        for (int t = 0; t < 2 * dim; ++t)
            if (gf.inside(i + dd[t][0], j + dd[t][1], k + dd[t][2]))
                a[oidx(dim, 1, dd[t][0], dd[t][1], dd[t][2])] = -scale * inv_h2;
    }
    return std::string();
}

std::string build_hierarchy(HostProblem& hp, int dim, int n, int n_levels, int scale_hd, int disc, const double* kappa2,
                            double kappa2_const, int m, const int32_t* obs_site, const double* obs_w,
                            int nnz_per_obs, const double* Gamma, const double* y, int* code)
{
    *code = MGMC_ERR_ARG;
    hp.dim = dim;
    hp.R = disc == 2 ? 2 : 1;
    hp.NS = dim == 2 ? (2 * hp.R + 1) * (2 * hp.R + 1) : 27;
    hp.C = (hp.NS - 1) / 2;
    hp.m = m;
    hp.scale_hd = scale_hd;
    hp.disc = disc;
    if (disc != 0 && disc != 1 && disc != 2) return "disc must be MGMC_FD, MGMC_Q1 or MGMC_SSL";
    if (disc == 1 && kappa2) return "the Q1 discretisation takes a constant kappa^2 (kappa2 = NULL)";
    if (disc == 2 && (kappa2 || dim != 2))
        return "the squared shifted Laplacian is 2D with a constant kappa^2 (kappa2 = NULL)";
    hp.n_levels = n_levels;
    hp.lev.assign(n_levels, HostLevel());
    {
        int nn = n;
        for (int l = n_levels - 1; l >= 0; --l) {
            hp.lev[l].n = nn;
            hp.lev[l].N = 1;
            for (int a = 0; a < dim; ++a) hp.lev[l].N *= nn;
            nn = (nn - 1) / 2;
        }
    }
    HostLevel& Fl = hp.lev[n_levels - 1];
    Grid gf{dim, n};
    // Gamma
    if (m > 0) {
        hp.Gamma.assign(Gamma, Gamma + (size_t)m * m);
        for (int i = 0; i < m; ++i) {
            if (!std::isfinite(y[i])) return "observed value y is not finite";
            for (int j = 0; j < m; ++j) {
                double a = hp.Gamma[(size_t)i * m + j], b = hp.Gamma[(size_t)j * m + i];
                if (!std::isfinite(a)) return "Gamma has a non-finite entry";
                if (std::fabs(a - b) > 1e-12 * (std::fabs(a) + std::fabs(b))) {
                    *code = MGMC_ERR_NOT_SPD;
                    return "Gamma is not symmetric";
                }
            }
        }
        std::vector<double> LG;
        if (!cholesky_lower(m, hp.Gamma, LG)) {
            *code = MGMC_ERR_NOT_SPD;
            return "Gamma is not positive definite";
        }
        if (!lu_inverse(m, hp.Gamma, hp.Gamma_inv)) {
            *code = MGMC_ERR_NOT_SPD;
            return "Gamma is singular";
        }
        hp.LG = LG;
        hp.gamma_diag = true;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < i; ++j)
                if (LG[(size_t)i * m + j] != 0.0) hp.gamma_diag = false;
        hp.y.assign(y, y + m);
    }
    // finest operator
    {
        std::string e = fine_operator(hp, dim, n, scale_hd, disc, kappa2, kappa2_const);
        if (!e.empty()) return e;
    }
    // fine B from the caller's rows
    Fl.bptr.assign(m + 1, 0);
    for (int k = 0; k < m; ++k) {
        std::map<long long, double> col;
        for (int t = 0; t < nnz_per_obs; ++t) {
            int s = obs_site[(size_t)k * nnz_per_obs + t];
            double w = obs_w[(size_t)k * nnz_per_obs + t];
            if (s < 0) continue;
            if (s >= Fl.N) return "observation site out of range";
            if (!std::isfinite(w)) return "observation weight is not finite";
            col[s] += w;
        }
        for (auto& kv : col) {
            Fl.bsite.push_back(kv.first);
            Fl.bw.push_back(kv.second);
        }
        Fl.bptr[k + 1] = (int)Fl.bsite.size();
    }
    // f_L norm: ||B Gamma^-1 y||
    if (m > 0) {
        std::vector<double> g(m, 0.0);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) g[i] += hp.Gamma_inv[(size_t)i * m + j] * y[j];
        std::map<long long, double> f;
        for (int k = 0; k < m; ++k)
            for (int t = Fl.bptr[k]; t < Fl.bptr[k + 1]; ++t) f[Fl.bsite[t]] += Fl.bw[t] * g[k];
        double s2 = 0.0;
        for (auto& kv : f) s2 += kv.second * kv.second;
        hp.f_norm = std::sqrt(s2);
    }
    // coarse levels
    for (int l = n_levels - 1; l >= 1; --l) {
        galerkin(hp, hp.lev[l], hp.lev[l - 1]);
        coarsen_B(hp, hp.lev[l], hp.lev[l - 1]);
    }
    for (int l = 0; l < n_levels; ++l) {
        HostLevel& L = hp.lev[l];
        for (long long s = 0; s < L.N; ++s)
            if (!(L.st[(size_t)s * hp.NS + hp.C] > 0.0)) {
                *code = MGMC_ERR_NOT_SPD;
                return "operator has a non-positive diagonal entry";
            }
    }
    for (int l = 1; l < n_levels; ++l)
        for (int dir = 0; dir < 2; ++dir)
            if (!lowrank_setup(hp, hp.lev[l], dir)) {
                *code = MGMC_ERR_NOT_SPD;
                return "Gamma + B^T M^-1 B is singular";
            }
    // coarsest posterior operator and its factor
    {
        HostLevel& L0 = hp.lev[0];
        int n0 = (int)L0.N;
        if (n0 > MGMC_MAX_COARSEST) return "coarsest grid too large: add levels";
        hp.n0 = n0;
        Grid g0{dim, L0.n};
        std::vector<double> A0((size_t)n0 * n0, 0.0);
        const int R = hp.R, rz = dim == 3 ? R : 0;
        for (int s = 0; s < n0; ++s) {
            int i, j, k;
            g0.coords(s, i, j, k);
            for (int oz = -rz; oz <= rz; ++oz)
                for (int oy = -R; oy <= R; ++oy)
                    for (int ox = -R; ox <= R; ++ox)
                        if (g0.inside(i + ox, j + oy, k + oz))
                            A0[(size_t)s * n0 + g0.idx(i + ox, j + oy, k + oz)] +=
                                L0.st[(size_t)s * hp.NS + oidx(dim, R, ox, oy, oz)];
        }
        if (m > 0) {
            // B_0 Gamma^-1 B_0^T
            std::vector<double> Bd((size_t)n0 * m, 0.0);
            for (int k = 0; k < m; ++k)
                for (int t = L0.bptr[k]; t < L0.bptr[k + 1]; ++t) Bd[(size_t)L0.bsite[t] * m + k] += L0.bw[t];
            for (int a = 0; a < n0; ++a)
                for (int b = 0; b < n0; ++b) {
                    double acc = 0.0;
                    for (int k = 0; k < m; ++k) {
                        if (Bd[(size_t)a * m + k] == 0.0) continue;
                        for (int t = 0; t < m; ++t)
                            acc += Bd[(size_t)a * m + k] * hp.Gamma_inv[(size_t)k * m + t] * Bd[(size_t)b * m + t];
                    }
                    A0[(size_t)a * n0 + b] += acc;
                }
        }
        if (!cholesky_lower(n0, A0, hp.chol0)) {
            *code = MGMC_ERR_NOT_SPD;
            return "coarsest posterior operator is not positive definite";
        }
    }
    *code = MGMC_OK;
    return std::string();
}

}  // namespace mgmc
