// Kernels of the earthquake location and origin-time gradients (tt_reloc.cu).
#pragma once

#include <cuda_runtime.h>

#include "tt_common.cuh"

namespace ttgb {

// Values and physical gradients of the trilinear interpolants of M batched fields G
// ([N][M], F) at n_pts points (double [n_pts][3]: depth km, lat deg, lon deg): val [n_pts][M],
// grad [n_pts][M][3]. *bad = 1 when a point lies outside the grid (its row then uses the
// clamped cell's lower corner; no access leaves the field).
template <typename F>
cudaError_t run_field_at_points(const GridC &g, int M, int n_pts, const void *G,
                                const double *pts, double *val, double *grad, int *bad,
                                cudaStream_t st);
// Kx [n_src][3] = sum_m R[n][m] grad[n][m], Kt [n_src] = sum_m R[n][m] (Eqs. B5-B11).
cudaError_t run_reloc_kernels(int n_src, int n_rec, const double *R, const double *grad,
                              double *Kx, double *Kt, cudaStream_t st);
// Bounds of the grid as given by the caller: depth km, latitude and longitude degrees.
struct GridBox {
    double lo[3], hi[3];
};
// Normalised gradient step of the event positions (clamped to box) and origin times.
cudaError_t run_reloc_update(const GridC &g, const GridBox &box, int n_src, double *pts,
                             double *otime, const double *Kx, const double *Kt, double step_km,
                             double step_s, cudaStream_t st);

}  // namespace ttgb
