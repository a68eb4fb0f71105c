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

// The region's solve itself is the node-hyperplane sweep (tt_sweep.cu) with SCHEME 3, on
// T - c_e: sign < 0 saves c_e = T[node 0][e] into c [n_ev] and subtracts it from every node of
// event e; sign > 0 adds it back.
template <typename F>
cudaError_t run_tele_shift(long long N, int n_ev, void *T, void *c, int sign, cudaStream_t st);

}  // namespace ttgb
