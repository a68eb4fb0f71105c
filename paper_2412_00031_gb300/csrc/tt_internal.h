// Host-side declarations shared by the translation units of libttgb.
#pragma once

#include <cuda.h>
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

// Tile schedule of one tile shape: tiles (I << 20 | J << 10 | K) grouped by I + J + K.
struct TileSchedule {
    unsigned int *tiles = nullptr;
    int *off = nullptr;
    int n_planes = 0;
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
    int scheme;                // local solver: 0 Lax-Friedrichs, 1 Godunov (isotropic models)
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
    // tile-wavefront schedule (fwd_tile_kernel): tiles of one sweep grouped by tile hyperplane
    const unsigned int *tiles;
    const int *toff;
    int n_tplanes;
    int na, nb, nc;   // interior extent swept
    int ngroups;      // groups of 32 sources
    // barrier groups of the node schedule: blocks [g * grp_blocks, (g + 1) * grp_blocks) solve
    // the sources [g * grp_src, min(B, (g + 1) * grp_src)) with their own barrier bar[g]
    int n_bgroups, grp_blocks, grp_src;
    // sources of this launch: [src_lo, src_lo + src_n); t0c caches 1/T0 and grad T0 / T0 of
    // the factor for them, [node][src_n]
    int src_lo, src_n;
    Vec4<F> *t0c;
    int idx32;        // every [node][source] index fits in 32 bits
    // Retire-and-refill mode (refill != 0): the launch works on B slots; tau and t0c are
    // the slots' working columns ([N][B]) and src their SrcC copies. Sources 0..n_all-1
    // come from a queue: when a slot's source converges (or reaches max_iter) its column is
    // copied to tau_out[N][n_all], and the slot takes the next source. iters / conv are
    // per source then ([n_all]).
    int refill, n_all, init_from_out;
    F *tau_out;
    const SrcC *src_all;                    // [n_all]
    const Vec2<F> *tabT_all, *tabP_all;     // [n_t][n_all], [n_p][n_all]
    SrcC *slot_srcc;                        // [B]
    int *slot_src, *slot_prev, *slot_it, *slot_fill, *queue;  // [B] each; queue: 1 int
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
    // Face coefficients, four planes of [N][B] (plane stride N * B): A a / delta on the +r,
    // +theta, +phi faces and J_c S_c (NaN on the source's fixed set)
    F *coef;
    int n_bgroups, grp_blocks, grp_src;  // barrier groups (as in FwdArgs)
    int grp_base;              // group index of this launch's first group
    const unsigned int *nodes;
    const int *off;
    BarrierState *bar;
    F *partial;                // [grid][2][B]: max |dP|, max |P| of the last sweep
    int *conv, *iters, *n_active;
    F tol;
    int max_iter;
    unsigned long long spin_ns;
};

// Dynamic shared memory of the node-hyperplane forward sweep: the per-source maxima of a
// barrier group, then (staged kernel) the two-stage copy buffers of every thread.
template <typename F> __host__ __device__ inline size_t fwd_err_bytes(int grp_src) {
    return ((size_t)grp_src * sizeof(F) + 127) / 128 * 128;
}
template <typename F> size_t fwd_smem_bytes(int grp_src, int block);

// Launchers (tt_sweep.cu). They return a cudaError_t of the launch itself.
template <typename F> cudaError_t launch_forward(const FwdArgs<F> &a, int grid, int block,
                                                 cudaStream_t st);
template <typename F> cudaError_t launch_adjoint(const AdjArgs<F> &a, int grid, int block,
                                                 cudaStream_t st);
template <typename F> int forward_blocks_per_sm(int block, size_t smem, bool idx32, int scheme = 0);
template <typename F> cudaError_t launch_t0_cache(const FwdArgs<F> &a, cudaStream_t st);
// Slot table of the retire-and-refill mode: slot s < n_slots takes source s.
template <typename F> cudaError_t launch_refill_setup(const FwdArgs<F> &a, cudaStream_t st);

// Tile shapes of the tile-wavefront forward sweep (sweep-local a = r, b = theta, c = phi).
struct TileShape {
    int ta, tb, tc;
};
constexpr int kNumTileShapes = 3;
constexpr TileShape kTileShapes[kNumTileShapes] = {{2, 4, 8}, {4, 4, 4}, {2, 8, 8}};
template <typename F> size_t forward_tiled_smem(int shape, int B);
template <typename F>
cudaError_t launch_forward_tiled(const CUtensorMap &map_tau, const CUtensorMap &map_rec,
                                 const CUtensorMap &map_t0c, const FwdArgs<F> &a, int shape,
                                 int grid, cudaStream_t st);
template <typename F> int forward_tiled_blocks_per_sm(int shape, int B);
constexpr int kTileThreads = 256;
// Sources one lane of the node-hyperplane forward sweep updates at each node (a warp covers
// 32 x this many consecutive sources); barrier groups are sized in multiples of a warp's.
#ifndef TTGB_FWD_NS
#define TTGB_FWD_NS 2
#endif
constexpr int kFwdSourcesPerLane = TTGB_FWD_NS;
constexpr int kMaxBarrierGroups = 8;
template <typename F> int adjoint_blocks_per_sm(int block, size_t smem);
// Face-coefficient adjoint: coefficients once per solve, then the sweep over P.
template <typename F> cudaError_t launch_adjoint_coefs(const AdjArgs<F> &a, cudaStream_t st);
template <typename F> cudaError_t launch_adjoint_faces(const AdjArgs<F> &a, int grid, int block,
                                                       cudaStream_t st);
template <typename F> int adjoint_faces_blocks_per_sm(int block, size_t smem);

}  // namespace ttgb
