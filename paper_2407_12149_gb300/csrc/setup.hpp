// setup.hpp -- host-side (FP64) construction of the MGMC hierarchy.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace mgmc {

struct HostLevel {
    int n = 0;
    long long N = 0;
    std::vector<double> st;          // [N * W^d] full stencil, W = 2R + 1, offset (dx+R) + W(dy+R) [+ W^2(dz+R)]
    // B_l by columns: entries bptr[k] .. bptr[k+1]-1 of (dense site, weight)
    std::vector<int> bptr;
    std::vector<long long> bsite;
    std::vector<double> bw;
    // G_l(dir) on its support
    std::vector<long long> gsite[2];
    std::vector<double> gval[2];     // [rows * m]
    // fused-path extras (forward direction): H = P^T A_l G_l on the coarse grid
    // (fixes the restricted residual after the low-rank correction) and
    // B_l^T G_l (m x m, row-major)
    std::vector<long long> hsite;    // coarse dense sites
    std::vector<double> hval;        // [rows * m]
    std::vector<double> BtG;
};

struct HostProblem {
    int dim = 2, NS = 9, C = 4;
    int R = 1;                        // stencil radius: 1, or 2 for the squared shifted Laplacian
    int n_levels = 1;
    int m = 0;
    int scale_hd = 1;
    int disc = 0;                     // finest grid: 0 finite differences, 1 Q1 elements, 2 squared shifted Laplacian
    double woff_fine = 0.0;           // s / h^2 of the finest grid
    std::vector<double> kappa_part;  // s * kappa^2 at the fine sites
    std::vector<HostLevel> lev;      // 0 = coarsest
    std::vector<double> Gamma, Gamma_inv, LG, y;
    bool gamma_diag = true;
    int n0 = 0;
    std::vector<double> chol0;       // Cholesky factor of A~_0 (lower, row-major)
    double f_norm = 0.0;             // ||f_L||_2
};

// Returns an empty string on success, otherwise an error message; *code gets
// the mgmc_status to return.
std::string build_hierarchy(HostProblem& hp, int dim, int n, int n_levels, int scale_hd, int disc, const double* kappa2,
                            double kappa2_const, int m, const int32_t* obs_site, const double* obs_w,
                            int nnz_per_obs, const double* Gamma, const double* y, int* code);

// The finest grid's operator alone: hp.dim, NS, C, n_levels and lev[] must be set
// (build_hierarchy does this); fills lev[n_levels - 1].st.
std::string fine_operator(HostProblem& hp, int dim, int n, int scale_hd, int disc, const double* kappa2,
                          double kappa2_const);

// H = P^T A_l G_l(forward) and B_l^T G_l(forward) for level l >= 1.
void fused_extras(HostLevel& L, const HostProblem& hp, int l);

// Row sums of a level's stencil (for the FP32 correction form).
std::vector<double> row_sums(const HostProblem& hp, int l);

}  // namespace mgmc
