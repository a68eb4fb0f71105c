// Kernels of teleseismic events (tt_tele.cu).
#pragma once

#include <cuda_runtime.h>

#include "tt_common.cuh"

namespace ttgb {

// 2-D traveltimes of n_ev events (one block each) on r = r_min + i dr, Delta = j dd:
// s_r [n_r] of F, r_src [n_ev] double, tau scratch and T [n_ev][n_r][n_d] of F, iters [n_ev].
template <typename F>
cudaError_t run_tele2d(int n_r, int n_d, double r_min, double dr, double dd, const void *s_r,
                       const double *r_src, int n_ev, double tol, int max_iter, void *tau,
                       void *T, int *iters, cudaStream_t st);
// The 2-D times interpolated at every node of the region: T [N][n_ev] of F; ev_ll [n_ev][2]
// the events' latitude and longitude in radians.
template <typename F>
cudaError_t run_region_times(const GridC &g, int n_r, int n_d, double r_min, double dr2,
                             double dd, const void *T2, int n_ev, const double *ev_ll, void *T,
                             cudaStream_t st);

// One hyperplane (ordering o; nodes[p0 .. p0 + cnt) of the interior schedule) of the region's
// Lax-Friedrichs solve of T with fixed faces: T [N][n_ev]; err_bits [n_ev] the largest change
// of each event (as double bits); events with done[e] are skipped.
template <typename F>
cudaError_t run_tele3d_plane(const GridC &g, const void *s, const void *xi, const void *eta,
                             const unsigned *nodes, int p0, int cnt, int o, int n_ev,
                             const int *done, void *T, unsigned long long *err_bits,
                             cudaStream_t st);

}  // namespace ttgb
