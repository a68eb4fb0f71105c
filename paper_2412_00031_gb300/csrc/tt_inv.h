// Kernels of the inversion step's regularisation and update (tt_inv.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace ttgb {

// Forward grid (nr x nt x np) and H inversion grids of cr x ct x cp nodes.
struct MgDims {
    int nr, nt, np;
    int cr, ct, cp;
    int H;
};

// Host tables of one axis: W[h][a][i] and lo[h][i] (tt_inv.cu).
void mgrid_axis_tables(int n, int c, int H, std::vector<double> &W, std::vector<int> &lo);

// Eqs. 4 and A4 over the entries of every (source, receiver) (see tt_inv.cu); *bad = 1 for
// an entry whose other source is out of range (the entry is skipped).
cudaError_t run_misfit_cr(int n_src, int n_rec, const int *off, const int *other,
                          const double *dtobs, const double *w, double gamma, const double *Tr,
                          double *chi, double *R, int *bad, cudaStream_t st);
// Kd[node] += sum over the B sources of P[node][b] (Eq. 19), FP64, a fixed order.
template <typename F>
cudaError_t run_kernel_density(long long N, int B, const F *P, double *Kd, cudaStream_t st);
// Eq. 18 in place.
cudaError_t run_kernel_normalize(long long N, double *Ks, double *Kxi, double *Keta,
                                 const double *Kd, double eps, double zeta, cudaStream_t st);
// Eq. 17: G[h][a][b][c] for one kernel K; T1 ([H][nr][nt][cp]) and T2 ([H][nr][ct][cp]) are
// scratch; dV = h2[i]^2 cost[j] dvol.
cudaError_t run_mgrid_project(const MgDims &d, const double *K, const double *h2,
                              const double *cost, double dvol, const double *Wr,
                              const double *Wt, const double *Wp, double *T1, double *T2,
                              double *G, cudaStream_t st);
// Eq. 15: D at the forward nodes from the coefficients G; lo = the three axes' lo tables.
cudaError_t run_mgrid_expand(const MgDims &d, const double *G, const int *lo, const double *Wr,
                             const double *Wt, const double *Wp, double *D, cudaStream_t st);
// Eq. 18 with eps = eps_rel max(Kd), the maximum taken on the device; part: scratch of
// 3 n_part + 3 doubles.
cudaError_t run_kernel_normalize_rel(long long N, double *Ks, double *Kxi, double *Keta,
                                     const double *Kd, double eps_rel, double zeta, double *part,
                                     int n_part, cudaStream_t st);
// *out = alpha sum chi[b][0] + beta sum chi[b][1] + gamma sum chi_cr[b] (chi_cr may be NULL),
// FP64 in a fixed order.
cudaError_t run_misfit_total(int n, const double *chi, double alpha, double beta,
                             const double *chi_cr, double gamma, double *out, cudaStream_t st);
// The model update; part: scratch of 3 n_part + 3 doubles.
template <typename F>
cudaError_t run_model_update(long long N, F *s, F *xi, F *eta, const double *Ds,
                             const double *Dxi, const double *Deta, double step, double *part,
                             int n_part, cudaStream_t st);

}  // namespace ttgb
