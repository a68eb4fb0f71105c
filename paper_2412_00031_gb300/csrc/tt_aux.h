// Host launchers of the set-up and non-sweep kernels (tt_aux.cu).
#pragma once

#include <cuda_runtime.h>

#include "tt.h"
#include "tt_common.cuh"

namespace ttgb {

struct PointD {  // same layout as tt_point
    double depth, lat, lon;
};

// Checks a grid description (3 < n <= TT_MAX_DIM per axis, ordered and non-empty extents,
// a radius above the deepest layer, a known geometry, and for spherical grids latitudes
// strictly inside (-89, 89) degrees, away from the poles where 1 / cos(theta) blows up) and
// fills the device constants. Returns false for an invalid grid. Every entry point that
// takes a tt_grid validates it here.
bool grid_constants(const tt_grid &G, GridC &g);

template <typename F>
cudaError_t run_source_setup(const GridC &g, const void *s, const void *xi, const void *eta,
                             const PointD *d_pts, int n_src, SrcC *d_src, Vec2<F> *tabT,
                             Vec2<F> *tabP, cudaStream_t st);
template <typename F>
cudaError_t run_node_records(const GridC &g, const void *s, const void *xi, const void *eta,
                             const double *h2, const double *cost, NodeRec<F> *rec, int *bad,
                             cudaStream_t st);
template <typename F>
cudaError_t run_tau_init(const GridC &g, int n_src, const SrcC *d_src, F *tau, bool fill,
                         cudaStream_t st);
// Batch order of a plan's forward (sources sorted by their previous iteration counts):
// perm = identity; perm = sources sorted by (iters, index); out[q] = in[perm[q]];
// tau_o[n][q] = tau[n][perm[q]] (to_order) or the reverse; a[perm[q]] = a_o[q] (and b);
// out[q][:] = in[perm[q]][:] for rows of n doubles.
cudaError_t run_order_identity(int B, int *perm, cudaStream_t st);
cudaError_t run_order_update(int B, const int *iters, int *perm, cudaStream_t st);
cudaError_t run_gather_points(int B, const int *perm, const PointD *in, PointD *out,
                              cudaStream_t st);
template <typename F>
cudaError_t run_permute_rows(long long N, int B, const int *perm, F *tau, F *tau_o, bool to_order,
                             cudaStream_t st);
cudaError_t run_unpermute_ints(int B, const int *perm, const int *a_o, const int *b_o, int *a,
                               int *b, cudaStream_t st);
cudaError_t run_gather_rows(int B, int n, const int *perm, const double *in, double *out,
                            cudaStream_t st);
// Fills tau [N][n_src] with the start from above of opts.init = 3 (twice a bound of tau
// from the model's slowness and anisotropy); hilo: 2 unsigned of device scratch.
template <typename F>
cudaError_t run_upper_start(const GridC &g, int n_src, const void *s, const void *xi,
                            const void *eta, F *tau, unsigned *hilo, cudaStream_t st);
template <typename F>
cudaError_t run_traveltime(const GridC &g, int B, const SrcC *src, const Vec2<F> *tabT,
                           const Vec2<F> *tabP, const F *rad, const F *cost, const F *sint,
                           const F *tau, F *T, cudaStream_t st);
cudaError_t run_receiver_setup(const GridC &g, const PointD *d_rec, int n_rec, long long *cq,
                               double *wq, int *bad, cudaStream_t st);
template <typename F>
cudaError_t run_point_sources(const GridC &g, int n_rec, const long long *cq, const double *wq,
                              int *sidx, int *next, int *heads, int *n_heads, const double *R,
                              int B, F *JS, cudaStream_t st);
template <typename F>
cudaError_t run_misfit(int B, int n_rec, const void *T, const long long *cq, const double *wq,
                       const tt_data &d, double *Tr, double *chi, double *R, int *bad,
                       cudaStream_t st);
// The same misfit from given receiver times: Tr[b][m] = tab[b][m] + otime[b] (otime may be
// NULL).
cudaError_t run_misfit_table(int B, int n_rec, const double *tab, const double *otime,
                             const tt_data &d, double *Tr, double *chi, double *R, int *bad,
                             cudaStream_t st);
template <typename F>
cudaError_t run_kernel_accum(const GridC &g, int B, const void *s, const void *T, const void *P,
                             const double *h2, const double *cost, double *Ks, double *Kxi,
                             double *Keta, int n_sm, cudaStream_t st);

}  // namespace ttgb
