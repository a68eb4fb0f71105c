// Host-side declarations shared by the translation units of libttgb.
#pragma once

#include <cuda_runtime.h>

#include "tt_common.cuh"

namespace ttgb {

// Schedule of one sweep: nodes grouped by hyperplane a + b + c = L (Sec. 3.4), each node
// packed as (a << 20) | (b << 10) | c in sweep-local coordinates; plane L occupies
// [off[L], off[L+1]).
struct Schedule {
    unsigned int *nodes = nullptr;
    int *off = nullptr;
    int n_planes = 0;
    int lo = 0;  // first swept index on every axis (1 = interior sweep, 0 = all nodes)
    int na = 0, nb = 0, nc = 0;
};

template <typename F> struct GeoTab {
    F *rad = nullptr;    // r_i
    F *cost = nullptr;   // cos theta_j   (flat: 1)
    F *sint = nullptr;   // sin theta_j   (flat: 0)
    F *costf = nullptr;  // cos theta_{j+1/2} (flat: 1)
    F *h2 = nullptr;     // metric factor of theta: r_i (flat: R_E); phi's is h2 * cos theta
    F *arf = nullptr;    // (r_i + dr/2)^2 (flat: R_E^2): r-face area over cos theta
};

template <typename F> struct FwdArgs {
    GridC g;
    int B, slots, n_planes;
    F er;                      // 1 / (2 dr)
    const NodeRec<F> *rec;
    F *tau;
    const SrcC *src;
    const Vec2<F> *tabT, *tabP;
    const F *rad, *cost, *sint;
    const unsigned int *nodes;
    const int *off;
    BarrierState *bar;
    F *partial;
    int *conv, *iters, *n_active;
    F tol;
    int max_iter;
    unsigned long long spin_ns;
};

template <typename F> struct AdjArgs {
    GridC g;
    int B, slots, n_planes, n_rec;
    const F *T;
    F *P;
    const F *xi, *eta;
    const SrcC *src;
    const F *cost, *costf, *h2, *arf;
    const int *sidx;           // [N] index into JS or kNone
    const F *JS;               // [n_heads][B] J_c S_c of Eq. 5's point sources
    const unsigned int *nodes;
    const int *off;
    BarrierState *bar;
    F *partial;                // [grid][2][B]: max |dP|, max |P| of the last sweep
    int *conv, *iters, *n_active;
    F tol;
    int max_iter;
    unsigned long long spin_ns;
};

// Launchers (tt_sweep.cu). They return a cudaError_t of the launch itself.
template <typename F> cudaError_t launch_forward(const FwdArgs<F> &a, int grid, int block,
                                                 cudaStream_t st);
template <typename F> cudaError_t launch_adjoint(const AdjArgs<F> &a, int grid, int block,
                                                 cudaStream_t st);
template <typename F> int forward_blocks_per_sm(int block, size_t smem);
template <typename F> int adjoint_blocks_per_sm(int block, size_t smem);

}  // namespace ttgb
