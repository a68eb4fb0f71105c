// C ABI of libttgb (declared in include/tt.h): context, validation, workspace and the
// orchestration of the kernels in tt_sweep.cu and tt_aux.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <vector>

#include "tt.h"
#include "tt_aux.h"
#include "tt_internal.h"
#include "tt_inv.h"
#include "tt_reloc.h"
#include "tt_tele.h"
#include "tt_net.h"

using namespace ttgb;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct tt_ctx {
    tt_grid grid;
    GridC g;
    cudaStream_t st = nullptr;
    int device = 0, n_sm = 0;
    char err[512] = {0};

    Schedule interior, full;
    TileSchedule tiled[kNumTileShapes];
    GeoTab<float> gf;
    GeoTab<double> gd;

    // workspace, grown on demand
    DevBuf src, pts, rpts, tabT, tabP, rec, partial, conv, iters, nact, bar, flags;
    DevBuf cq, wq, sidx, next, heads, nheads, JS, coef, t0c;
    // warm-start network: inference weights (BF16-rounded) and its workspace
    DevBuf net_theta, net_x, net_a, net_b, net_y, net_d1, net_d2, net_dy, net_wt, net_part,
        net_scr, net_wbf;  // net_wbf: BF16 weight images of the four layers (tensor cores)
    // tensor-core training: weight images of theta and of the transposed layers, BF16 rows
    DevBuf net_img, net_timg, net_rows;
    bool has_net = false;
    int net_stride = 1;        // the warm-start network's grid: every net_stride-th node
    double *h_loss = nullptr;  // pinned
    // autotuner: scratch tau and the choices made, per (n_src, dtype)
    DevBuf tune_tau, tau_w, slot_srcc, slot_int;
    // batch order of single forward calls: the last iteration counts of recent source sets
    // (keyed by a hash of the positions) and the ordered batch's buffers
    struct OrderMemo {
        unsigned long long key;
        int B;
        std::vector<int> iters;
    };
    std::vector<OrderMemo> order_memo;
    DevBuf ord_perm, ord_pts, ord_src, ord_tabT, ord_tabP, ord_tau, ord_iters, ord_conv;
    // inversion step: multiple-grid tables (for mg_key), projection scratch, update scratch
    DevBuf mg_tab, mg_scr, upd_part;
    // teleseismic events: 2-D tau scratch, event radii / coordinates and iteration counts
    DevBuf tele_tau, tele_aux;
    int mg_key[4] = {0, 0, 0, 0};
    struct Tuned { int n_src, dtype, scheme, schedule, groups; };
    std::vector<Tuned> tuned;
    struct TunedAdj { int n_src, dtype, chunk, groups; };
    std::vector<TunedAdj> tuned_adj;
    int *h_pinned = nullptr;  // readback: [0..TT_MAX_BATCH) iterations, then flags
    PointD *h_pts = nullptr;  // staging for source / receiver positions
    size_t h_pts_cap = 0;

    cudaEvent_t ev_start[2] = {nullptr, nullptr}, ev_stop[2] = {nullptr, nullptr};
    cudaEvent_t ev_net[2] = {nullptr, nullptr};  // around the warm-start inference
    cudaEvent_t ev_kacc[2] = {nullptr, nullptr}; // around the last kernel accumulation
    int kacc_B = 0;                              // its source count
    bool warm_last = false;                      // the last forward used the warm start
    int scheme_last = 0;                         // local solver of the last forward
    tt_stats stats[3] = {};
    long long launches = 0;   // kernels launched by this context
};

namespace {

constexpr long long kDefaultSpinNs = 2000000000LL;
// Device flags of a context or plan: [0] model, [1] data index, [2] receiver position,
// [3] network wait (read back after each call); [4], [5] the start-from-above bound.
constexpr int kFlagInts = 6;
// Largest per-(node, source) coefficient array the adjoint keeps in its workspace.
constexpr size_t kCoefBudgetBytes = 64ull << 30;
// Largest factor cache (1/T0 and grad T0 / T0 per node and source) one forward slice keeps.
constexpr size_t kFactorCacheBudgetBytes = 32ull << 30;
// Barrier groups that one face-adjoint launch runs side by side.
#ifndef TTGB_ADJ_GROUPS
#define TTGB_ADJ_GROUPS 4
#endif
constexpr int kAdjGroups = TTGB_ADJ_GROUPS;

tt_status fail(tt_ctx *c, tt_status s, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(ctx, TT_ECUDA, "%s (line %d) failed: %s", #call, __LINE__,   \
                        cudaGetErrorString(e_));                                      \
    } while (0)

tt_status ensure(tt_ctx *ctx, DevBuf &b, size_t bytes) {
    if (bytes <= b.bytes) return TT_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, TT_ENOMEM, "workspace allocation of %zu bytes failed", want);
    }
    b.bytes = want;
    return TT_OK;
}

#define ENSURE(buf, bytes)                        \
    do {                                          \
        tt_status s_ = ensure(ctx, buf, (bytes)); \
        if (s_ != TT_OK) return s_;               \
    } while (0)

bool inside(const tt_ctx *ctx, const tt_point &p) {
    const tt_grid &G = ctx->grid;
    const double eps = 1e-9;
    double span_d = G.depth_max_km - G.depth_min_km;
    double span_t = G.lat_max_deg - G.lat_min_deg, span_p = G.lon_max_deg - G.lon_min_deg;
    return std::isfinite(p.depth_km) && std::isfinite(p.lat_deg) && std::isfinite(p.lon_deg) &&
           p.depth_km >= G.depth_min_km - eps * span_d &&
           p.depth_km <= G.depth_max_km + eps * span_d &&
           p.lat_deg >= G.lat_min_deg - eps * span_t && p.lat_deg <= G.lat_max_deg + eps * span_t &&
           p.lon_deg >= G.lon_min_deg - eps * span_p && p.lon_deg <= G.lon_max_deg + eps * span_p;
}

tt_status build_schedule(tt_ctx *ctx, Schedule &S, int lo) {
    const GridC &g = ctx->g;
    S.lo = lo;
    S.na = g.nr - 2 * lo;
    S.nb = g.nt - 2 * lo;
    S.nc = g.np - 2 * lo;
    S.n_planes = S.na + S.nb + S.nc - 2;
    std::vector<unsigned int> nodes;
    nodes.reserve((size_t)S.na * S.nb * S.nc);
    std::vector<int> off(S.n_planes + 1, 0);
    for (int L = 0; L < S.n_planes; ++L) {
        off[L] = (int)nodes.size();
        for (int a = 0; a < S.na; ++a) {
            if (a > L) break;
            for (int b = 0; b < S.nb; ++b) {
                int c = L - a - b;
                if (c < 0) break;
                if (c >= S.nc) continue;
                nodes.push_back(((unsigned)a << 20) | ((unsigned)b << 10) | (unsigned)c);
            }
        }
    }
    off[S.n_planes] = (int)nodes.size();
    CK(cudaMalloc((void **)&S.nodes, nodes.size() * sizeof(unsigned int)));
    CK(cudaMalloc((void **)&S.off, off.size() * sizeof(int)));
    CK(cudaMemcpy(S.nodes, nodes.data(), nodes.size() * sizeof(unsigned int),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(S.off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    return TT_OK;
}

tt_status build_tile_schedule(tt_ctx *ctx, TileSchedule &S, const TileShape &sh) {
    const GridC &g = ctx->g;
    const int nI = (g.nr - 2 + sh.ta - 1) / sh.ta, nJ = (g.nt - 2 + sh.tb - 1) / sh.tb;
    const int nK = (g.np - 2 + sh.tc - 1) / sh.tc;
    S.n_planes = nI + nJ + nK - 2;
    std::vector<unsigned int> tiles;
    std::vector<int> off(S.n_planes + 1, 0);
    for (int L = 0; L < S.n_planes; ++L) {
        off[L] = (int)tiles.size();
        for (int I = 0; I < nI && I <= L; ++I)
            for (int J = 0; J < nJ && I + J <= L; ++J) {
                int K = L - I - J;
                if (K < nK) tiles.push_back(((unsigned)I << 20) | ((unsigned)J << 10) | (unsigned)K);
            }
    }
    off[S.n_planes] = (int)tiles.size();
    CK(cudaMalloc((void **)&S.tiles, tiles.size() * sizeof(unsigned int)));
    CK(cudaMalloc((void **)&S.off, off.size() * sizeof(int)));
    CK(cudaMemcpy(S.tiles, tiles.data(), tiles.size() * sizeof(unsigned int),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(S.off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    return TT_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// 4-D tiled tensor map over an [n_r][n_t][n_p][inner] array of F (inner innermost).
template <typename F>
tt_status encode_map4(tt_ctx *ctx, CUtensorMap *map, const void *base, long long inner,
                      const unsigned box[4]) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(ctx, TT_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    const GridC &g = ctx->g;
    const cuuint64_t es = sizeof(F);
    cuuint64_t dims[4] = {(cuuint64_t)inner, (cuuint64_t)g.np, (cuuint64_t)g.nt, (cuuint64_t)g.nr};
    cuuint64_t strides[3] = {inner * es, (cuuint64_t)g.np * inner * es,
                             (cuuint64_t)g.nt * g.np * inner * es};
    cuuint32_t boxd[4] = {box[0], box[1], box[2], box[3]};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, sizeof(F) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                     4, const_cast<void *>(base), dims, strides, boxd, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, TT_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TT_OK;
}

template <typename F>
tt_status upload_tab(tt_ctx *ctx, F *&dst, const std::vector<double> &v) {
    std::vector<F> tmp(v.begin(), v.end());
    CK(cudaMalloc((void **)&dst, tmp.size() * sizeof(F)));
    CK(cudaMemcpy(dst, tmp.data(), tmp.size() * sizeof(F), cudaMemcpyHostToDevice));
    return TT_OK;
}

template <typename F> tt_status upload_geo(tt_ctx *ctx, GeoTab<F> &t) {
    const GridC &g = ctx->g;
    std::vector<double> rad(g.nr), cost(g.nt), sint(g.nt), costf(g.nt), h2(g.nr), arf(g.nr);
    for (int i = 0; i < g.nr; ++i) {
        double r = g.r0 + i * g.dr, rf = r + 0.5 * g.dr;
        rad[i] = r;
        h2[i] = g.flat ? g.re : r;
        arf[i] = g.flat ? g.re * g.re : rf * rf;
    }
    for (int j = 0; j < g.nt; ++j) {
        double th = g.t0 + j * g.dt;
        cost[j] = g.flat ? 1.0 : std::cos(th);
        sint[j] = g.flat ? 0.0 : std::sin(th);
        costf[j] = g.flat ? 1.0 : std::cos(th + 0.5 * g.dt);
    }
    tt_status s;
    if ((s = upload_tab<F>(ctx, t.rad, rad)) != TT_OK) return s;
    if ((s = upload_tab<F>(ctx, t.cost, cost)) != TT_OK) return s;
    if ((s = upload_tab<F>(ctx, t.sint, sint)) != TT_OK) return s;
    if ((s = upload_tab<F>(ctx, t.costf, costf)) != TT_OK) return s;
    if ((s = upload_tab<F>(ctx, t.h2, h2)) != TT_OK) return s;
    return upload_tab<F>(ctx, t.arf, arf);
}

template <typename F> void free_geo(GeoTab<F> &t) {
    F *ps[] = {t.rad, t.cost, t.sint, t.costf, t.h2, t.arf};
    for (F *p : ps)
        if (p) cudaFree(p);
}

// Launch shape of a persistent sweep: as many co-resident blocks as useful (at most two per
// SM), never more threads than the widest hyperplane needs.
template <typename F>
tt_status sweep_shape(tt_ctx *ctx, bool fwd, int B, const Schedule &S, int cap, int &grid,
                      int &block, int &slots) {
    block = sizeof(F) == 4 ? 512 : 256;
    size_t smem = (size_t)B * sizeof(F) * (fwd ? 1 : 2);
    int per_sm = fwd ? forward_blocks_per_sm<F>(block, smem, false)
                     : adjoint_blocks_per_sm<F>(block, smem);
    if (per_sm <= 0) return fail(ctx, TT_ECUDA, "sweep kernel cannot be resident (B = %d)", B);
    if (per_sm > 2) per_sm = 2;
    long long max_grid = (long long)per_sm * ctx->n_sm;
    long long widest = 0;
    // widest plane: bounded by the two largest axis extents
    long long d[3] = {S.na, S.nb, S.nc};
    for (int x = 0; x < 3; ++x)
        for (int y = x + 1; y < 3; ++y) widest = d[x] * d[y] > widest ? d[x] * d[y] : widest;
    long long want = (widest * B + block - 1) / block;
    long long min_grid = ((long long)B + block - 1) / block;
    if (want < min_grid) want = min_grid;
    if (cap > 0 && cap < max_grid) max_grid = cap;
    grid = (int)(want < max_grid ? want : max_grid);
    if ((long long)grid * block < B)
        return fail(ctx, TT_EINVAL, "batch of %d sources exceeds one resident launch", B);
    slots = (int)(((long long)grid * block) / B);
    return TT_OK;
}

tt_status check_model(tt_ctx *ctx, const tt_model *m) {
    if (!m || !m->d_s || !m->d_xi || !m->d_eta)
        return fail(ctx, TT_EINVAL, "model pointers must be non-NULL");
    if (m->dtype != TT_F32 && m->dtype != TT_F64)
        return fail(ctx, TT_EINVAL, "model dtype %d is neither TT_F32 nor TT_F64", m->dtype);
    return TT_OK;
}

tt_status check_sources(tt_ctx *ctx, const tt_point *h_src, int n_src) {
    if (n_src < 1 || n_src > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "n_src = %d outside 1..%d", n_src, TT_MAX_BATCH);
    if (!h_src) return fail(ctx, TT_EINVAL, "source array is NULL");
    for (int b = 0; b < n_src; ++b)
        if (!inside(ctx, h_src[b]))
            return fail(ctx, TT_EINVAL, "source %d (%g km, %g, %g) outside the grid", b,
                        h_src[b].depth_km, h_src[b].lat_deg, h_src[b].lon_deg);
    return TT_OK;
}

tt_status check_opts(tt_ctx *ctx, const tt_opts *o) {
    if (!o) return fail(ctx, TT_EINVAL, "opts is NULL");
    if (!(o->tol_fwd > 0) || !(o->tol_adj > 0) || o->max_iter_fwd < 1 || o->max_iter_adj < 1)
        return fail(ctx, TT_EINVAL, "tolerances must be > 0 and iteration limits >= 1");
    if (o->sweep_schedule < 0 || o->sweep_schedule > 1 + kNumTileShapes)
        return fail(ctx, TT_EINVAL, "sweep_schedule %d unknown", o->sweep_schedule);
    if (o->init < 0 || o->init > 3) return fail(ctx, TT_EINVAL, "init %d unknown", o->init);
    if (o->scheme < 0 || o->scheme > 2) return fail(ctx, TT_EINVAL, "scheme %d unknown", o->scheme);
    if (o->fwd_slots < 0) return fail(ctx, TT_EINVAL, "fwd_slots %d < 0", o->fwd_slots);
    if (o->fwd_groups < 0 || o->fwd_groups > kMaxBarrierGroups)
        return fail(ctx, TT_EINVAL, "fwd_groups %d outside 0..%d", o->fwd_groups,
                    kMaxBarrierGroups);
    if (o->adj_groups < 0 || o->adj_groups > kMaxBarrierGroups)
        return fail(ctx, TT_EINVAL, "adj_groups %d outside 0..%d", o->adj_groups,
                    kMaxBarrierGroups);
    if (o->adj_chunk < 0) return fail(ctx, TT_EINVAL, "adj_chunk %d < 0", o->adj_chunk);
    if (o->fwd_order < 0 || o->fwd_order > 1)
        return fail(ctx, TT_EINVAL, "fwd_order %d is not 0 or 1", o->fwd_order);
    if (o->init == 2 && !ctx->has_net)
        return fail(ctx, TT_EINVAL, "init = 2 (warm start) needs tt_net_set_weights first");
    return TT_OK;
}

unsigned long long spin_ns(const tt_opts *o) {
    return (unsigned long long)(o->spin_limit_ns > 0 ? o->spin_limit_ns : kDefaultSpinNs);
}

// Device buffers of one solve step. A context call fills it from the context's grow-on-demand
// workspace; a plan (tt_plan) owns its buffers for the plan's lifetime.
template <typename F> struct Work {
    PointD *src_pts = nullptr, *rec_pts = nullptr;
    SrcC *src = nullptr;
    Vec2<F> *tabT = nullptr, *tabP = nullptr;
    NodeRec<F> *rec = nullptr;
    Vec4<F> *t0c = nullptr, *coef = nullptr;
    F *partial = nullptr;
    int *conv_f = nullptr, *iters_f = nullptr, *conv_a = nullptr, *iters_a = nullptr;
    int *nact = nullptr, *flags = nullptr;  // flags: model, data index, receiver position
    BarrierState *bar = nullptr;
    long long *cq = nullptr;
    double *wq = nullptr;
    int *sidx = nullptr, *next = nullptr, *heads = nullptr, *nheads = nullptr;
    F *JS = nullptr;
    int t0c_slice = 0;  // sources per forward slice the factor cache holds
    // retire-and-refill forward: slot working columns and slot table
    F *tau_w = nullptr;
    SrcC *slot_srcc = nullptr;
    int *slot_int = nullptr;  // slot_src, slot_prev, slot_it, slot_fill ([slots] each), queue
    int n_slots = 0;
    bool coef_ok = false;
    // warm start: features [chunk][N][6], activations [chunk][N][32] (two), output [chunk][N]
    float *net_x = nullptr, *net_y = nullptr;
    __nv_bfloat16 *net_a = nullptr, *net_b = nullptr;   // BF16 activations
    const float *net_theta = nullptr;
    const __nv_bfloat16 *net_wbf = nullptr;
    int net_chunk = 0;
};

// The warm-start network's grid (net_grid_of with the context's stride), its extent as
// convolution dimensions, and its node count.
NetGrid net_grid(const tt_ctx *ctx) { return net_grid_of(ctx->g, ctx->net_stride); }
ConvDims net_dims(const tt_ctx *ctx, int nb) {
    const NetGrid n = net_grid(ctx);
    return ConvDims{nb, n.nr, n.nt, n.np};
}
long long net_nodes(const tt_ctx *ctx) {
    const NetGrid n = net_grid(ctx);
    return (long long)n.nr * n.nt * n.np;
}

// Rows of one network grid in the padded row layout of the tensor-core inference.
size_t net_grid_rows(const tt_ctx *ctx) { return net_rows(net_dims(ctx, 1)); }

// Sources per warm-start inference pass: two BF16 activation buffers of at most ~8 GB
// together, and at most 64 sources.
int net_chunk(const tt_ctx *ctx, int B) {
    const size_t per_src = net_grid_rows(ctx) * kNetHidden * sizeof(__nv_bfloat16);
    long long c = (long long)((4ull << 30) / per_src);
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return (int)(c < B ? c : B);
}

int factor_slice(const GridC &g, int B, size_t es) {
    const size_t per_src = 4 * es * (size_t)g.N;
    if (per_src * (size_t)B <= kFactorCacheBudgetBytes) return B;
    int slice = (int)(kFactorCacheBudgetBytes / per_src) / 32 * 32;
    return slice < 32 ? 32 : slice;
}

size_t partial_bytes(const tt_ctx *ctx, int B, size_t es) {
    return 2 * es * (size_t)B * (size_t)(kMaxBarrierGroups * ctx->n_sm);
}

// Fills W from the context workspace for a step over B sources and n_rec receivers (0 for
// a forward-only call).
template <typename F> tt_status work_from_ctx(tt_ctx *ctx, Work<F> &W, int B, int n_rec) {
    const GridC &g = ctx->g;
    const int slice = factor_slice(g, B, sizeof(F));
    ENSURE(ctx->src, sizeof(SrcC) * (size_t)B);
    ENSURE(ctx->tabT, sizeof(Vec2<F>) * (size_t)g.nt * B);
    ENSURE(ctx->tabP, sizeof(Vec2<F>) * (size_t)g.np * B);
    ENSURE(ctx->rec, sizeof(NodeRec<F>) * (size_t)g.N);
    ENSURE(ctx->t0c, sizeof(Vec4<F>) * (size_t)g.N * slice);
    ENSURE(ctx->partial, partial_bytes(ctx, B, sizeof(F)));
    ENSURE(ctx->conv, sizeof(int) * (size_t)B);
    ENSURE(ctx->iters, sizeof(int) * (size_t)B);
    ENSURE(ctx->nact, sizeof(int) * kMaxBarrierGroups);
    ENSURE(ctx->bar, sizeof(BarrierState) * kMaxBarrierGroups);
    ENSURE(ctx->flags, kFlagInts * sizeof(int));
    W.src = (SrcC *)ctx->src.p;
    W.tabT = (Vec2<F> *)ctx->tabT.p;
    W.tabP = (Vec2<F> *)ctx->tabP.p;
    W.rec = (NodeRec<F> *)ctx->rec.p;
    W.t0c = (Vec4<F> *)ctx->t0c.p;
    W.t0c_slice = slice;
    W.partial = (F *)ctx->partial.p;
    W.conv_f = W.conv_a = (int *)ctx->conv.p;
    W.iters_f = W.iters_a = (int *)ctx->iters.p;
    W.nact = (int *)ctx->nact.p;
    W.bar = (BarrierState *)ctx->bar.p;
    W.flags = (int *)ctx->flags.p;
    W.src_pts = (PointD *)ctx->pts.p;
    if (n_rec > 0) {
        const int S = 8 * n_rec;
        ENSURE(ctx->cq, sizeof(long long) * S);
        ENSURE(ctx->wq, sizeof(double) * S);
        ENSURE(ctx->sidx, sizeof(int) * (size_t)g.N);
        ENSURE(ctx->next, sizeof(int) * S);
        ENSURE(ctx->heads, sizeof(int) * S);
        ENSURE(ctx->nheads, sizeof(int));
        ENSURE(ctx->JS, sizeof(F) * (size_t)S * B);
        W.cq = (long long *)ctx->cq.p;
        W.wq = (double *)ctx->wq.p;
        W.sidx = (int *)ctx->sidx.p;
        W.next = (int *)ctx->next.p;
        W.heads = (int *)ctx->heads.p;
        W.nheads = (int *)ctx->nheads.p;
        W.JS = (F *)ctx->JS.p;
        const size_t coef_bytes = sizeof(Vec4<F>) * (size_t)g.N * B;
        W.coef_ok = coef_bytes <= kCoefBudgetBytes;
        if (W.coef_ok) {
            ENSURE(ctx->coef, coef_bytes);
            W.coef = (Vec4<F> *)ctx->coef.p;
        }
    }
    return TT_OK;
}

// Slots of the retire-and-refill forward (0: every source resident): opts->fwd_slots
// rounded up to a multiple of 32, at most the factor cache's slice.
int refill_slots_for(const tt_opts *o, int B, int slice) {
    if (o->fwd_slots <= 0 || o->fwd_slots >= B) return 0;
    int S = (o->fwd_slots + 31) / 32 * 32;
    if (S > slice) S = slice / 32 * 32;
    return S >= B ? 0 : S;
}

template <typename F> tt_status refill_work_from_ctx(tt_ctx *ctx, Work<F> &W, int S) {
    ENSURE(ctx->tau_w, sizeof(F) * (size_t)ctx->g.N * S);
    ENSURE(ctx->slot_srcc, sizeof(SrcC) * (size_t)S);
    ENSURE(ctx->slot_int, sizeof(int) * (4 * (size_t)S + 1));
    W.tau_w = (F *)ctx->tau_w.p;
    W.slot_srcc = (SrcC *)ctx->slot_srcc.p;
    W.slot_int = (int *)ctx->slot_int.p;
    W.n_slots = S;
    return TT_OK;
}

// Warm-start inference buffers from the context workspace.
template <typename F> tt_status net_work_from_ctx(tt_ctx *ctx, Work<F> &W, int B) {
    const int c = net_chunk(ctx, B);
    const size_t Nn = (size_t)net_nodes(ctx);
    ENSURE(ctx->net_x, sizeof(float) * kNetFeatures * Nn * c);
    ENSURE(ctx->net_a, sizeof(__nv_bfloat16) * kNetHidden * net_grid_rows(ctx) * c);
    ENSURE(ctx->net_b, sizeof(__nv_bfloat16) * kNetHidden * net_grid_rows(ctx) * c);
    ENSURE(ctx->net_y, sizeof(float) * Nn * c);
    W.net_x = (float *)ctx->net_x.p;
    W.net_a = (__nv_bfloat16 *)ctx->net_a.p;
    W.net_b = (__nv_bfloat16 *)ctx->net_b.p;
    W.net_y = (float *)ctx->net_y.p;
    W.net_theta = (const float *)ctx->net_theta.p;
    W.net_wbf = (const __nv_bfloat16 *)ctx->net_wbf.p;
    W.net_chunk = c;
    return TT_OK;
}

// Host positions -> pinned staging -> device (synchronises the stream first: the staging
// buffer may still be read by an earlier call).
tt_status stage_to(tt_ctx *ctx, const tt_point *h, int n, PointD *d) {
    if ((size_t)n > ctx->h_pts_cap) {
        if (ctx->h_pts) cudaFreeHost(ctx->h_pts);
        ctx->h_pts = nullptr;
        ctx->h_pts_cap = 0;
        CK(cudaMallocHost((void **)&ctx->h_pts, sizeof(PointD) * (size_t)n));
        ctx->h_pts_cap = n;
    }
    CK(cudaStreamSynchronize(ctx->st));
    for (int q = 0; q < n; ++q) ctx->h_pts[q] = PointD{h[q].depth_km, h[q].lat_deg, h[q].lon_deg};
    CK(cudaMemcpyAsync(d, ctx->h_pts, sizeof(PointD) * (size_t)n, cudaMemcpyHostToDevice, ctx->st));
    return TT_OK;
}

template <typename F> GeoTab<F> &geo(tt_ctx *ctx);
template <> GeoTab<float> &geo<float>(tt_ctx *ctx) { return ctx->gf; }
template <> GeoTab<double> &geo<double>(tt_ctx *ctx) { return ctx->gd; }

// ---------------------------------------------------------------- enqueue-only steps
// Each enqueues kernels and memsets on ctx->st and nothing else: no synchronisation and no
// host access, so that a whole step can be captured into a CUDA graph.

// Timing events: while the stream is being captured, a plain record is only a dependency
// marker, so the record becomes an event node of the graph instead.
cudaError_t record(tt_ctx *ctx, cudaEvent_t ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(ctx->st, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(ev, ctx->st, cudaEventRecordExternal)
               : cudaEventRecord(ev, ctx->st);
}

template <typename F>
tt_status enq_sources(tt_ctx *ctx, Work<F> &W, const tt_model *m, int B) {
    CK(run_source_setup<F>(ctx->g, m->d_s, m->d_xi, m->d_eta, W.src_pts, B, W.src, W.tabT,
                           W.tabP, ctx->st));
    ctx->launches += 3;
    return TT_OK;
}

// Network forward over d.nb grids: x (6 channels) -> a1 -> a2 -> a3 -> y. For inference
// a3 may alias a1.
tt_status enq_net_forward(tt_ctx *ctx, const float *theta, const float *x, const ConvDims &d,
                          float *a1, float *a2, float *a3, float *y) {
    const float *in = x;
    float *outs[kNetLayers] = {a1, a2, a3, y};
    for (int l = 0; l < kNetLayers; ++l) {
        const float *w = theta + net_weight_offset(l);
        const float *bias = w + 27 * kNetCin[l] * kNetCout[l];
        CK(run_conv3d(d, kNetCin[l], kNetCout[l], in, l > 0, w, bias, nullptr, outs[l], ctx->st));
        in = outs[l];
    }
    ctx->launches += kNetLayers;
    return TT_OK;
}

// tau = 1 + clamp(net(features), -0.5, 1) for every source, in chunks of W.net_chunk, the
// network evaluated on its grid (net_grid) and interpolated to every node when coarser. A
// device-side wait of the tensor-core kernels that exceeds spin sets flags[3].
template <typename F>
tt_status enq_warm_start(tt_ctx *ctx, Work<F> &W, const tt_model *m, int B, F *tau,
                         unsigned long long spin) {
    const GridC &g = ctx->g;
    const NetGrid ng = net_grid(ctx);
    const GeoTab<F> &t = geo<F>(ctx);
    for (int b0 = 0; b0 < B; b0 += W.net_chunk) {
        const int nb = W.net_chunk < B - b0 ? W.net_chunk : B - b0;
        CK(run_net_features<F>(g, ng, B, b0, nb, W.src, W.tabT, W.tabP, t.rad, t.cost,
                               (const F *)m->d_s, (const F *)m->d_xi, (const F *)m->d_eta,
                               W.net_x, ctx->st));
        CK(run_net_infer(net_dims(ctx, nb), W.net_theta, W.net_wbf, W.net_x, W.net_a, W.net_b,
                         W.net_y, ctx->n_sm, W.flags + 3, spin, ctx->st));
        CK(run_warm_tau<F>(g, ng, B, b0, nb, W.net_y, tau, ctx->st));
        ctx->launches += 3 + kNetLayers;
    }
    return TT_OK;
}

template <typename F>
tt_status enq_forward(tt_ctx *ctx, Work<F> &W, const tt_model *m, int B, void *d_tau,
                      void *d_T, const tt_opts *o) {
    const GridC &g = ctx->g;
    tt_status s;
    CK(cudaMemsetAsync(W.conv_f, 0, sizeof(int) * (size_t)B, ctx->st));
    CK(cudaMemsetAsync(W.iters_f, 0, sizeof(int) * (size_t)B, ctx->st));
    CK(cudaMemsetAsync(W.nact, 0, sizeof(int) * kMaxBarrierGroups, ctx->st));
    CK(cudaMemsetAsync(W.bar, 0, sizeof(BarrierState) * kMaxBarrierGroups, ctx->st));
    CK(cudaMemsetAsync(W.flags, 0, sizeof(int), ctx->st));
    CK(run_node_records<F>(g, m->d_s, m->d_xi, m->d_eta, ctx->gd.h2, ctx->gd.cost, W.rec,
                           W.flags, ctx->st));
    if (o->init == 2) {
        CK(record(ctx, ctx->ev_net[0]));
        CK(cudaMemsetAsync(W.flags + 3, 0, sizeof(int), ctx->st));
        if ((s = enq_warm_start<F>(ctx, W, m, B, (F *)d_tau, spin_ns(o))) != TT_OK) return s;
        CK(record(ctx, ctx->ev_net[1]));
    }
    if (o->init == 3)
        CK(run_upper_start<F>(g, B, m->d_s, m->d_xi, m->d_eta, (F *)d_tau,
                              (unsigned *)(W.flags + 4), ctx->st));
    CK(run_tau_init<F>(g, B, W.src, (F *)d_tau, o->init == 0, ctx->st));
    ctx->launches += 1 + (o->init == 0 ? 2 : o->init == 3 ? 3 : 1);

    // Tile schedules stage 32 sources per task with TMA: they need B >= 32 and rows of tau
    // (B values) that are a multiple of 16 bytes. Automatic: node hyperplanes.
    const bool tiles_ok = B >= 32 && (B * sizeof(F)) % 16 == 0;
    int sched = o->sweep_schedule == 0 ? 1 : o->sweep_schedule;
    if ((sched >= 2 && !tiles_ok) || W.n_slots > 0 || o->scheme != 0) sched = 1;
    const int slice = W.t0c_slice;

    const GeoTab<F> &t = geo<F>(ctx);
    FwdArgs<F> a;
    memset(&a, 0, sizeof a);
    a.g = g;
    a.B = B;
    a.scheme = o->scheme;
    a.n_planes = ctx->interior.n_planes;
    a.er = (F)(0.5 / g.dr);
    a.rec = W.rec;
    a.tau = (F *)d_tau;
    a.src = W.src;
    a.tabT = W.tabT;
    a.tabP = W.tabP;
    a.rad = t.rad;
    a.cost = t.cost;
    a.sint = t.sint;
    a.nodes = ctx->interior.nodes;
    a.off = ctx->interior.off;
    a.bar = W.bar;
    a.partial = W.partial;
    a.conv = W.conv_f;
    a.iters = W.iters_f;
    a.n_active = W.nact;
    a.tol = (F)o->tol_fwd;
    a.max_iter = o->max_iter_fwd;
    a.spin_ns = spin_ns(o);
    a.t0c = W.t0c;
    a.na = g.nr - 2;
    a.nb = g.nt - 2;
    a.nc = g.np - 2;
    a.idx32 = (unsigned long long)g.N * (unsigned long long)(B > 8 ? B : 8) < (1ull << 32);
    CUtensorMap map_tau, map_rec;
    if (sched >= 2) {
        const TileShape sh = kTileShapes[sched - 2];
        const unsigned box_tau[4] = {32u, (unsigned)sh.tc + 2, (unsigned)sh.tb + 2,
                                     (unsigned)sh.ta + 2};
        const unsigned box_rec[4] = {8u, (unsigned)sh.tc, (unsigned)sh.tb, (unsigned)sh.ta};
        if ((s = encode_map4<F>(ctx, &map_tau, d_tau, B, box_tau)) != TT_OK) return s;
        if ((s = encode_map4<F>(ctx, &map_rec, W.rec, 8, box_rec)) != TT_OK) return s;
        const TileSchedule &ts = ctx->tiled[sched - 2];
        a.tiles = ts.tiles;
        a.toff = ts.off;
        a.n_tplanes = ts.n_planes;
    }

    int max_grid_used = 0;
    CK(record(ctx, ctx->ev_start[TT_STATS_FORWARD]));
    if (W.n_slots > 0) {
        // Retire-and-refill: one launch over S slots; converged sources hand their slot to
        // the next queued source (each source's arithmetic is that of the resident launch).
        const int S = W.n_slots;
        a.refill = 1;
        a.n_all = B;
        a.init_from_out = o->init != 0;
        a.tau_out = (F *)d_tau;
        a.tau = W.tau_w;
        a.B = S;
        a.src_all = W.src;
        a.tabT_all = W.tabT;
        a.tabP_all = W.tabP;
        a.slot_srcc = W.slot_srcc;
        a.src = W.slot_srcc;
        a.slot_src = W.slot_int;
        a.slot_prev = W.slot_int + S;
        a.slot_it = W.slot_int + 2 * S;
        a.slot_fill = W.slot_int + 3 * S;
        a.queue = W.slot_int + 4 * S;
        a.src_lo = 0;
        a.src_n = S;
        a.idx32 = (unsigned long long)g.N * (unsigned long long)(S > 8 ? S : 8) < (1ull << 32);
        const int block = 256;
        int per_sm = forward_blocks_per_sm<F>(block, fwd_smem_bytes<F>(S, block), a.idx32 != 0,
                                              a.scheme);
        if (per_sm <= 0) return fail(ctx, TT_ECUDA, "sweep kernel cannot be resident");
        if (per_sm > kMaxBarrierGroups) per_sm = kMaxBarrierGroups;
        int max_grid = per_sm * ctx->n_sm;
        if (o->launch_blocks > 0 && o->launch_blocks < max_grid) max_grid = o->launch_blocks;
        int groups = o->fwd_groups > 0 ? o->fwd_groups : per_sm;
        if (groups > kMaxBarrierGroups) groups = kMaxBarrierGroups;
        const int wsrc = 32 * kFwdSourcesPerLane;
        if (groups > (S + wsrc - 1) / wsrc) groups = (S + wsrc - 1) / wsrc;
        if (groups > max_grid) groups = max_grid;
        int gsrc = ((S + groups - 1) / groups + wsrc - 1) / wsrc * wsrc;
        groups = (S + gsrc - 1) / gsrc;
        int gblocks = max_grid / groups;
        if ((long long)gblocks * block < gsrc) gblocks = (gsrc + block - 1) / block;
        if ((long long)gblocks * groups > (long long)per_sm * ctx->n_sm)
            return fail(ctx, TT_EINVAL, "%d slots exceed one resident launch", S);
        a.n_bgroups = groups;
        a.grp_blocks = gblocks;
        a.grp_src = gsrc;
        CK(launch_refill_setup<F>(a, ctx->st));
        CK(launch_forward<F>(a, gblocks * groups, block, ctx->st));
        ctx->stats[TT_STATS_FORWARD].block_threads = block;
        ctx->launches += 2;
        max_grid_used = gblocks * groups;
    }
    for (int s0 = 0; s0 < (W.n_slots > 0 ? 0 : B); s0 += slice) {
        const int n = slice < B - s0 ? slice : B - s0;
        a.src_lo = s0;
        a.src_n = n;
        int grid = 0;
        if (sched == 1 || n < 32) {  // a tile task stages 32 sources: short slices use nodes
            // 256-thread blocks; one barrier group per resident block slot of an SM, so
            // each SM interleaves the groups; each group gets a multiple of 32 sources.
            const int block = 256;
            int per_sm = forward_blocks_per_sm<F>(block, fwd_smem_bytes<F>(n, block), a.idx32 != 0,
                                                  a.scheme);
            if (per_sm <= 0) return fail(ctx, TT_ECUDA, "sweep kernel cannot be resident");
            if (per_sm > kMaxBarrierGroups) per_sm = kMaxBarrierGroups;
            int max_grid = per_sm * ctx->n_sm;
            if (o->launch_blocks > 0 && o->launch_blocks < max_grid) max_grid = o->launch_blocks;
            const int wsrc = 32 * kFwdSourcesPerLane;  // sources of one warp
            int groups = o->fwd_groups > 0 ? o->fwd_groups : per_sm;
            if (groups > kMaxBarrierGroups) groups = kMaxBarrierGroups;
            if (groups > (n + wsrc - 1) / wsrc) groups = (n + wsrc - 1) / wsrc;
            if (groups > max_grid) groups = max_grid;
            int gsrc = ((n + groups - 1) / groups + wsrc - 1) / wsrc * wsrc;
            groups = (n + gsrc - 1) / gsrc;
            int gblocks = max_grid / groups;
            if ((long long)gblocks * block < gsrc) {
                int need = (gsrc + block - 1) / block;
                if ((long long)need * groups > (long long)per_sm * ctx->n_sm)
                    return fail(ctx, TT_EINVAL, "slice of %d sources exceeds one resident launch", n);
                gblocks = need;
            }
            grid = gblocks * groups;
            a.n_bgroups = groups;
            a.grp_blocks = gblocks;
            a.grp_src = gsrc;
            CK(launch_t0_cache<F>(a, ctx->st));
            CK(launch_forward<F>(a, grid, block, ctx->st));
            ctx->stats[TT_STATS_FORWARD].block_threads = block;
        } else {
            int per_sm = forward_tiled_blocks_per_sm<F>(sched - 2, B);
            if (per_sm <= 0) return fail(ctx, TT_ECUDA, "tiled sweep cannot be resident");
            if (per_sm > 4) per_sm = 4;
            grid = per_sm * ctx->n_sm;
            if (o->launch_blocks > 0 && o->launch_blocks < grid) grid = o->launch_blocks;
            if ((long long)grid * kTileThreads < n) {
                int need = (n + kTileThreads - 1) / kTileThreads;
                if (need > per_sm * ctx->n_sm)
                    return fail(ctx, TT_EINVAL, "slice of %d sources exceeds one resident launch", n);
                grid = need;
            }
            a.slots = (int)(((long long)grid * kTileThreads) / n);
            a.ngroups = (n + 31) / 32;
            a.n_bgroups = 1;
            a.grp_blocks = grid;
            a.grp_src = n;
            CUtensorMap map_t0c;
            const TileShape sh = kTileShapes[sched - 2];
            const unsigned box_c[4] = {128u, (unsigned)sh.tc, (unsigned)sh.tb, (unsigned)sh.ta};
            if ((s = encode_map4<F>(ctx, &map_t0c, W.t0c, 4LL * n, box_c)) != TT_OK) return s;
            CK(launch_t0_cache<F>(a, ctx->st));
            CK(launch_forward_tiled<F>(map_tau, map_rec, map_t0c, a, sched - 2, grid, ctx->st));
            ctx->stats[TT_STATS_FORWARD].block_threads = kTileThreads;
        }
        ctx->launches += 2;
        if (grid > max_grid_used) max_grid_used = grid;
    }
    CK(record(ctx, ctx->ev_stop[TT_STATS_FORWARD]));
    ctx->stats[TT_STATS_FORWARD].grid_blocks = max_grid_used;
    if (d_T) {
        CK(run_traveltime<F>(g, B, W.src, W.tabT, W.tabP, t.rad, t.cost, t.sint, (const F *)d_tau,
                             (F *)d_T, ctx->st));
        ctx->launches += 1;
    }
    return TT_OK;
}

// The forward over the batch in the order perm (perm[q] = the source at position q): the
// ordered batch gets its own source set-up (Wo: points, SrcC, angle tables, counts) and tau
// (tau_o); tau and the counts then go back to the batch's order (d_tau, W's counts) and T is
// computed from them. Each source's arithmetic does not depend on its position, so the
// results are those of the given order.
template <typename F>
tt_status enq_forward_ordered(tt_ctx *ctx, Work<F> &W, Work<F> &Wo, const int *perm,
                              const tt_model *m, int B, void *d_tau, void *tau_o, void *d_T,
                              const tt_opts *o) {
    const GridC &g = ctx->g;
    tt_status s;
    CK(run_gather_points(B, perm, W.src_pts, Wo.src_pts, ctx->st));
    if ((s = enq_sources<F>(ctx, Wo, m, B)) != TT_OK) return s;
    if (o->init == 1) CK(run_permute_rows<F>(g.N, B, perm, (F *)d_tau, (F *)tau_o, true, ctx->st));
    if ((s = enq_forward<F>(ctx, Wo, m, B, tau_o, nullptr, o)) != TT_OK) return s;
    CK(run_permute_rows<F>(g.N, B, perm, (F *)d_tau, (F *)tau_o, false, ctx->st));
    CK(run_unpermute_ints(B, perm, Wo.iters_f, Wo.conv_f, W.iters_f, W.conv_f, ctx->st));
    ctx->launches += 3 + (o->init == 1);
    if (d_T) {
        const GeoTab<F> &t = geo<F>(ctx);
        CK(run_traveltime<F>(g, B, W.src, W.tabT, W.tabP, t.rad, t.cost, t.sint, (const F *)d_tau,
                             (F *)d_T, ctx->st));
        ctx->launches += 1;
    }
    return TT_OK;
}

tt_status enq_receivers(tt_ctx *ctx, const PointD *rec_pts, int n_rec, long long *cq,
                        double *wq, int *flags) {
    CK(run_receiver_setup(ctx->g, rec_pts, n_rec, cq, wq, flags + 2, ctx->st));
    ctx->launches += 1;
    return TT_OK;
}

tt_status enq_misfit(tt_ctx *ctx, const void *d_T, int dtype, const tt_data *d,
                     const long long *cq, const double *wq, int *flags, double *d_Tr,
                     double *d_chi, double *d_R) {
    int *bad = flags + 1;
    if (dtype == TT_F32)
        CK(run_misfit<float>(d->n_src, d->n_rec, d_T, cq, wq, *d, d_Tr, d_chi, d_R, bad, ctx->st));
    else
        CK(run_misfit<double>(d->n_src, d->n_rec, d_T, cq, wq, *d, d_Tr, d_chi, d_R, bad, ctx->st));
    ctx->launches += 1;
    return TT_OK;
}

template <typename F>
tt_status enq_adjoint(tt_ctx *ctx, Work<F> &W, const tt_model *m, int B, const void *d_T,
                      int n_rec, const double *d_R, void *d_P, const tt_opts *o) {
    const GridC &g = ctx->g;
    tt_status s;
    CK(cudaMemsetAsync(W.conv_a, 0, sizeof(int) * (size_t)B, ctx->st));
    CK(cudaMemsetAsync(W.iters_a, 0, sizeof(int) * (size_t)B, ctx->st));
    CK(cudaMemsetAsync(W.nact, 0, sizeof(int) * kMaxBarrierGroups, ctx->st));
    CK(cudaMemsetAsync(W.bar, 0, sizeof(BarrierState) * kMaxBarrierGroups, ctx->st));
    CK(run_point_sources<F>(g, n_rec, W.cq, W.wq, W.sidx, W.next, W.heads, W.nheads, d_R, B, W.JS,
                            ctx->st));
    ctx->launches += 5;
    CK(cudaMemsetAsync(d_P, 0, sizeof(F) * (size_t)g.N * B, ctx->st));

    // Face-coefficient sweep when the per-(node, source) coefficients fit the workspace
    // budget; otherwise the sweep that evaluates the flux velocities at every update.
    const bool faces = W.coef_ok;
    int grid, block, slots;
    int n_bgroups = 1, grp_blocks = 0, grp_src = B, adj_launch_groups = 1;
    if (faces) {
        // Source slices of adj_chunk sources, one cooperative launch each, run one after
        // another: a hyperplane of one slice (coefficients of two planes, P of three) then
        // stays in L2. Automatic: slices of at most 128 sources.
        // Each launch covers `chunk` sources (default: all), split into up to
        // TTGB_ADJ_GROUPS barrier groups of >= 64 sources that run side by side.
        block = 256;
        int chunk = o->adj_chunk > 0 ? o->adj_chunk : B;
        chunk = chunk >= B ? B : (chunk + 31) / 32 * 32;
        int groups = o->adj_groups > 0 ? o->adj_groups : (chunk + 63) / 64;
        if (o->adj_groups <= 0 && groups > kAdjGroups) groups = kAdjGroups;
        if (groups > (chunk + 31) / 32) groups = (chunk + 31) / 32;  // >= 32 sources a group
        grp_src = ((chunk + groups - 1) / groups + 31) / 32 * 32;
        groups = (chunk + grp_src - 1) / grp_src;
        n_bgroups = (B + grp_src - 1) / grp_src;  // groups over the whole batch
        adj_launch_groups = groups;
        size_t smem = (size_t)grp_src * 2 * sizeof(F);
        int per_sm = adjoint_faces_blocks_per_sm<F>(block, smem);
        if (per_sm <= 0) return fail(ctx, TT_ECUDA, "adjoint sweep cannot be resident");
        if (per_sm > 4) per_sm = 4;
        int max_grid = per_sm * ctx->n_sm;
        if (o->launch_blocks > 0 && o->launch_blocks < max_grid) max_grid = o->launch_blocks;
        grp_blocks = max_grid / groups;
        if ((long long)grp_blocks * block < grp_src) {
            int need = (grp_src + block - 1) / block;
            if ((long long)need * groups > (long long)per_sm * ctx->n_sm)
                return fail(ctx, TT_EINVAL, "batch of %d sources exceeds one resident launch", B);
            grp_blocks = need;
        }
        grid = grp_blocks * groups;
        slots = 0;
    } else if ((s = sweep_shape<F>(ctx, false, B, ctx->full, o->launch_blocks, grid, block,
                                   slots)) != TT_OK) {
        return s;
    }
    const GeoTab<F> &t = geo<F>(ctx);
    AdjArgs<F> a;
    memset(&a, 0, sizeof a);
    a.g = g;
    a.B = B;
    a.slots = slots;
    a.n_planes = ctx->full.n_planes;
    a.n_rec = n_rec;
    a.T = (const F *)d_T;
    a.P = (F *)d_P;
    a.xi = (const F *)m->d_xi;
    a.eta = (const F *)m->d_eta;
    a.src = W.src;
    a.cost = t.cost;
    a.costf = t.costf;
    a.h2 = t.h2;
    a.arf = t.arf;
    a.sidx = W.sidx;
    a.JS = W.JS;
    a.nodes = ctx->full.nodes;
    a.off = ctx->full.off;
    a.bar = W.bar;
    a.partial = W.partial;
    a.conv = W.conv_a;
    a.iters = W.iters_a;
    a.n_active = W.nact;
    a.tol = (F)o->tol_adj;
    a.max_iter = o->max_iter_adj;
    a.spin_ns = spin_ns(o);
    a.coef = faces ? reinterpret_cast<F *>(W.coef) : nullptr;
    a.n_bgroups = n_bgroups;
    a.grp_blocks = grp_blocks;
    a.grp_src = grp_src;
    if (faces) {
        CK(launch_adjoint_coefs<F>(a, ctx->st));
        ctx->launches += 1;
    }
    CK(record(ctx, ctx->ev_start[TT_STATS_ADJOINT]));
    if (faces) {
        for (int q = 0; q < n_bgroups; q += adj_launch_groups) {
            a.grp_base = q;
            const int ng = n_bgroups - q < adj_launch_groups ? n_bgroups - q : adj_launch_groups;
            CK(launch_adjoint_faces<F>(a, grp_blocks * ng, block, ctx->st));
            ctx->launches += 1;
        }
    } else {
        CK(launch_adjoint<F>(a, grid, block, ctx->st));
        ctx->launches += 1;
    }
    CK(record(ctx, ctx->ev_stop[TT_STATS_ADJOINT]));
    ctx->stats[TT_STATS_ADJOINT].grid_blocks = grid;
    ctx->stats[TT_STATS_ADJOINT].block_threads = block;
    return TT_OK;
}

tt_status enq_kernel(tt_ctx *ctx, const tt_model *m, int B, const void *d_T, const void *d_P,
                     double *Ks, double *Kxi, double *Keta) {
    CK(record(ctx, ctx->ev_kacc[0]));
    ctx->kacc_B = B;
    if (m->dtype == TT_F32)
        CK(run_kernel_accum<float>(ctx->g, B, m->d_s, d_T, d_P, ctx->gd.h2, ctx->gd.cost, Ks, Kxi,
                                   Keta, ctx->n_sm, ctx->st));
    else
        CK(run_kernel_accum<double>(ctx->g, B, m->d_s, d_T, d_P, ctx->gd.h2, ctx->gd.cost, Ks,
                                    Kxi, Keta, ctx->n_sm, ctx->st));
    CK(record(ctx, ctx->ev_kacc[1]));
    ctx->launches += 1;
    return TT_OK;
}

// ---------------------------------------------------------------- read-back

// Nodes a source updates per sweep: the swept box minus the part of its 3x3x3 fixed set
// inside that box.
long long updated_nodes(const tt_ctx *ctx, const PointD &p, int lo) {
    const GridC &g = ctx->g;
    const double deg = 3.14159265358979323846 / 180.0;
    double f[3] = {((g.re - p.depth) - g.r0) / g.dr, (p.lat * deg - g.t0) / g.dt,
                   (p.lon * deg - g.p0) / g.dp};
    int n[3] = {g.nr, g.nt, g.np};
    long long box = 1, fixed = 1;
    for (int a = 0; a < 3; ++a) {
        int c = (int)std::floor(f[a] + 0.5);
        c = c < 0 ? 0 : (c > n[a] - 1 ? n[a] - 1 : c);
        int l0 = c - 1 > lo ? c - 1 : lo, l1 = c + 1 < n[a] - 1 - lo ? c + 1 : n[a] - 1 - lo;
        fixed *= l1 >= l0 ? (l1 - l0 + 1) : 0;
        box *= n[a] - 2 * lo;
    }
    return box - fixed;
}

// Host copy of the state a step leaves on the device.
struct Readback {
    int *iters_f, *conv_f, *iters_a, *conv_a;  // [TT_MAX_BATCH] each
    int *flags;                                // [4]
    unsigned char *bar_f, *bar_a;              // barrier words after the forward / adjoint
};

Readback readback_view(tt_ctx *ctx) {
    Readback r;
    r.iters_f = ctx->h_pinned;
    r.conv_f = ctx->h_pinned + TT_MAX_BATCH;
    r.iters_a = ctx->h_pinned + 2 * TT_MAX_BATCH;
    r.conv_a = ctx->h_pinned + 3 * TT_MAX_BATCH;
    r.flags = ctx->h_pinned + 4 * TT_MAX_BATCH;
    r.bar_f = (unsigned char *)(ctx->h_pinned + 4 * TT_MAX_BATCH + 8);
    r.bar_a = r.bar_f + sizeof(BarrierState) * kMaxBarrierGroups;
    return r;
}

// Pinned read-back buffer: the solves' state (readback_view), then one 64-byte slot for the
// scalar results of the reductions (tt_misfit_total).
size_t pinned_state_bytes() {
    const size_t b = sizeof(int) * (4 * TT_MAX_BATCH + 8) + 2 * sizeof(BarrierState) * kMaxBarrierGroups;
    return (b + 63) / 64 * 64;
}
size_t pinned_bytes() { return pinned_state_bytes() + 64; }
double *pinned_scalar(tt_ctx *ctx) {
    return reinterpret_cast<double *>(reinterpret_cast<char *>(ctx->h_pinned) + pinned_state_bytes());
}

// Enqueues the copies of one solve's state (forward or adjoint) into the pinned buffer.
tt_status enq_readback(tt_ctx *ctx, int B, const int *iters, const int *conv, const int *flags,
                       const BarrierState *bar, int which) {
    Readback r = readback_view(ctx);
    int *hi = which == TT_STATS_FORWARD ? r.iters_f : r.iters_a;
    int *hc = which == TT_STATS_FORWARD ? r.conv_f : r.conv_a;
    CK(cudaMemcpyAsync(hi, iters, sizeof(int) * (size_t)B, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(hc, conv, sizeof(int) * (size_t)B, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(r.flags, flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(which == TT_STATS_FORWARD ? r.bar_f : r.bar_a, bar,
                       sizeof(BarrierState) * kMaxBarrierGroups, cudaMemcpyDeviceToHost, ctx->st));
    return TT_OK;
}

// After the stream has finished: statuses of one solve and its statistics. src are the
// host positions of the sources (for the update counts).
tt_status solve_status(tt_ctx *ctx, int B, const PointD *src, int *h_iters, int max_iter,
                       const char *what, int which) {
    Readback r = readback_view(ctx);
    const int *hi = which == TT_STATS_FORWARD ? r.iters_f : r.iters_a;
    const int *hc = which == TT_STATS_FORWARD ? r.conv_f : r.conv_a;
    if (which == TT_STATS_FORWARD && (r.flags[0] & 1))
        return fail(ctx, TT_EINVAL, "%s: model has s <= 0 or xi^2 + eta^2 >= 1/4", what);
    if (which == TT_STATS_FORWARD && ctx->scheme_last == 1 && (r.flags[0] & 2))
        return fail(ctx, TT_EINVAL, "%s: the Godunov solver needs an isotropic model (xi = eta = 0)",
                    what);
    if (which == TT_STATS_FORWARD && ctx->warm_last && r.flags[3])
        return fail(ctx, TT_ETIMEOUT, "%s: a device-side wait of the warm start exceeded its limit",
                    what);
    for (int q = 0; q < kMaxBarrierGroups; ++q) {
        int st;
        const unsigned char *bar = which == TT_STATS_FORWARD ? r.bar_f : r.bar_a;
        memcpy(&st, bar + q * sizeof(BarrierState) + offsetof(BarrierState, status), sizeof st);
        if (st == kDevTimeout)
            return fail(ctx, TT_ETIMEOUT, "%s: a device-side wait exceeded its limit", what);
    }
    if (h_iters) memcpy(h_iters, hi, sizeof(int) * (size_t)B);
    tt_stats &S = ctx->stats[which];
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev_start[which], ctx->ev_stop[which]));
    S.sweep_ms = ms;
    S.warm_ms = 0.0;
    if (which == TT_STATS_FORWARD && ctx->warm_last) {
        CK(cudaEventElapsedTime(&ms, ctx->ev_net[0], ctx->ev_net[1]));
        S.warm_ms = ms;
    }
    const int lo = which == TT_STATS_FORWARD ? 1 : 0;
    long long upd = 0;
    int imax = 0;
    for (int b = 0; b < B; ++b) {
        upd += 8LL * hi[b] * updated_nodes(ctx, src[b], lo);
        imax = hi[b] > imax ? hi[b] : imax;
    }
    const GridC &g = ctx->g;
    S.node_updates = upd;
    S.iters_max = imax;
    S.node_sweeps = 8LL * imax * (long long)(g.nr - 2 * lo) * (g.nt - 2 * lo) * (g.np - 2 * lo);
    int nc = 0;
    for (int b = 0; b < B; ++b) nc += hc[b] == 0;
    if (nc)
        return fail(ctx, TT_ENOTCONVERGED, "%s: %d of %d sources did not converge in %d iterations",
                    what, nc, B, max_iter);
    return TT_OK;
}

// ---------------------------------------------------------------- immediate calls

// FNV-1a hash of a batch's source positions and dtype: the key of its remembered counts. A
// collision only changes the order of a sweep, never its results.
unsigned long long source_set_key(const tt_point *h_src, int B, int dtype) {
    unsigned long long h = 1469598103934665603ull ^ (unsigned long long)dtype;
    const unsigned char *p = reinterpret_cast<const unsigned char *>(h_src);
    for (size_t i = 0; i < sizeof(tt_point) * (size_t)B; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Keeps the forward iteration counts of the last solve of a source set (at most 64 sets).
void remember_counts(tt_ctx *ctx, unsigned long long key, int B, const int *iters) {
    for (auto &e : ctx->order_memo)
        if (e.key == key && e.B == B) {
            e.iters.assign(iters, iters + B);
            return;
        }
    if (ctx->order_memo.size() >= 64) ctx->order_memo.erase(ctx->order_memo.begin());
    ctx->order_memo.push_back(tt_ctx::OrderMemo{key, B, std::vector<int>(iters, iters + B)});
}

template <typename F>
tt_status forward_impl(tt_ctx *ctx, const tt_model *m, const tt_point *h_src, int B, void *d_tau,
                       void *d_T, const tt_opts *o, int *h_iters) {
    tt_status s;
    ENSURE(ctx->pts, sizeof(PointD) * (size_t)B);
    Work<F> W;
    if ((s = work_from_ctx<F>(ctx, W, B, 0)) != TT_OK) return s;
    if (o->init == 2 && (s = net_work_from_ctx<F>(ctx, W, B)) != TT_OK) return s;
    const int S = refill_slots_for(o, B, W.t0c_slice);
    if (S > 0 && (s = refill_work_from_ctx<F>(ctx, W, S)) != TT_OK) return s;
    if ((s = stage_to(ctx, h_src, B, W.src_pts)) != TT_OK) return s;
    if ((s = enq_sources<F>(ctx, W, m, B)) != TT_OK) return s;
    // the batch order: the last counts of the same source set, fewest first
    const unsigned long long key = source_set_key(h_src, B, m->dtype);
    const std::vector<int> *prev = nullptr;
    if (o->fwd_order == 0 && S == 0 && B >= 64)
        for (const auto &e : ctx->order_memo)
            if (e.key == key && e.B == B) prev = &e.iters;
    if (prev) {
        std::vector<int> perm(B);
        for (int q = 0; q < B; ++q) perm[q] = q;
        std::stable_sort(perm.begin(), perm.end(),
                         [prev](int a, int b) { return (*prev)[a] < (*prev)[b]; });
        ENSURE(ctx->ord_perm, sizeof(int) * (size_t)B);
        ENSURE(ctx->ord_pts, sizeof(PointD) * (size_t)B);
        ENSURE(ctx->ord_src, sizeof(SrcC) * (size_t)B);
        ENSURE(ctx->ord_tabT, sizeof(Vec2<F>) * (size_t)ctx->g.nt * B);
        ENSURE(ctx->ord_tabP, sizeof(Vec2<F>) * (size_t)ctx->g.np * B);
        ENSURE(ctx->ord_tau, sizeof(F) * (size_t)ctx->g.N * B);
        ENSURE(ctx->ord_iters, sizeof(int) * (size_t)B);
        ENSURE(ctx->ord_conv, sizeof(int) * (size_t)B);
        CK(cudaMemcpyAsync(ctx->ord_perm.p, perm.data(), sizeof(int) * (size_t)B,
                           cudaMemcpyHostToDevice, ctx->st));
        Work<F> Wo = W;
        Wo.src_pts = (PointD *)ctx->ord_pts.p;
        Wo.src = (SrcC *)ctx->ord_src.p;
        Wo.tabT = (Vec2<F> *)ctx->ord_tabT.p;
        Wo.tabP = (Vec2<F> *)ctx->ord_tabP.p;
        Wo.iters_f = (int *)ctx->ord_iters.p;
        Wo.conv_f = (int *)ctx->ord_conv.p;
        if ((s = enq_forward_ordered<F>(ctx, W, Wo, (const int *)ctx->ord_perm.p, m, B, d_tau,
                                        ctx->ord_tau.p, d_T, o)) != TT_OK)
            return s;
        // the host copy of perm must outlive the copy above
        CK(cudaStreamSynchronize(ctx->st));
    } else if ((s = enq_forward<F>(ctx, W, m, B, d_tau, d_T, o)) != TT_OK) {
        return s;
    }
    if ((s = enq_readback(ctx, B, W.iters_f, W.conv_f, W.flags, W.bar, TT_STATS_FORWARD)) != TT_OK)
        return s;
    CK(cudaStreamSynchronize(ctx->st));
    ctx->warm_last = o->init == 2;
    ctx->scheme_last = o->scheme;
    const tt_status st = solve_status(ctx, B, ctx->h_pts, h_iters, o->max_iter_fwd, "tt_forward",
                                      TT_STATS_FORWARD);
    if ((st == TT_OK || st == TT_ENOTCONVERGED) && o->fwd_order == 0 && S == 0 && B >= 64)
        remember_counts(ctx, key, B, readback_view(ctx).iters_f);
    return st;
}

template <typename F>
tt_status adjoint_impl(tt_ctx *ctx, const tt_model *m, const tt_point *h_src, int B,
                       const void *d_T, int n_rec, const tt_point *h_rec, const double *d_R,
                       void *d_P, const tt_opts *o, int *h_iters) {
    tt_status s;
    ENSURE(ctx->pts, sizeof(PointD) * (size_t)(B > n_rec ? B : n_rec));
    ENSURE(ctx->rpts, sizeof(PointD) * (size_t)n_rec);
    Work<F> W;
    if ((s = work_from_ctx<F>(ctx, W, B, n_rec)) != TT_OK) return s;
    W.rec_pts = (PointD *)ctx->rpts.p;
    CK(cudaMemsetAsync(W.flags, 0, 4 * sizeof(int), ctx->st));
    if ((s = stage_to(ctx, h_rec, n_rec, W.rec_pts)) != TT_OK) return s;
    if ((s = enq_receivers(ctx, W.rec_pts, n_rec, W.cq, W.wq, W.flags)) != TT_OK) return s;
    if ((s = stage_to(ctx, h_src, B, W.src_pts)) != TT_OK) return s;
    if ((s = enq_sources<F>(ctx, W, m, B)) != TT_OK) return s;
    if ((s = enq_adjoint<F>(ctx, W, m, B, d_T, n_rec, d_R, d_P, o)) != TT_OK) return s;
    if ((s = enq_readback(ctx, B, W.iters_a, W.conv_a, W.flags, W.bar, TT_STATS_ADJOINT)) != TT_OK)
        return s;
    CK(cudaStreamSynchronize(ctx->st));
    if (readback_view(ctx).flags[2])
        return fail(ctx, TT_EINVAL, "tt_adjoint: receiver outside the grid");
    return solve_status(ctx, B, ctx->h_pts, h_iters, o->max_iter_adj, "tt_adjoint",
                        TT_STATS_ADJOINT);
}

tt_status check_data(tt_ctx *ctx, const tt_data *d) {
    if (!d || !d->d_abs_off || !d->d_cs_off || !d->h_rec)
        return fail(ctx, TT_EINVAL, "data: NULL argument");
    if (d->n_src < 1 || d->n_src > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "n_src = %d outside 1..%d", d->n_src, TT_MAX_BATCH);
    if (d->n_rec < 1) return fail(ctx, TT_EINVAL, "need at least one receiver");
    if ((size_t)d->n_rec * 2 * 4 * sizeof(double) > 200 * 1024)
        return fail(ctx, TT_EINVAL, "n_rec = %d too large for the misfit kernel", d->n_rec);
    for (int q = 0; q < d->n_rec; ++q)
        if (!inside(ctx, d->h_rec[q]))
            return fail(ctx, TT_EINVAL, "receiver %d (%g km, %g, %g) outside the grid", q,
                        d->h_rec[q].depth_km, d->h_rec[q].lat_deg, d->h_rec[q].lon_deg);
    return TT_OK;
}

}  // namespace

extern "C" {

void tt_default_opts(tt_opts *o, int dtype) {
    if (!o) return;
    double tol = dtype == TT_F64 ? 1e-8 : 1e-6;
    o->tol_fwd = tol;
    o->tol_adj = tol;
    o->max_iter_fwd = 500;
    o->max_iter_adj = 500;
    o->init = 0;
    o->spin_limit_ns = 0;
    o->launch_blocks = 0;
    o->sweep_schedule = 0;
    o->adj_chunk = 0;
    o->fwd_groups = 0;
    o->fwd_slots = 0;
    o->scheme = 0;
    o->adj_groups = 0;
    o->fwd_order = 0;
}

const char *tt_last_error(const tt_ctx *ctx) { return ctx ? ctx->err : "no context"; }

tt_status tt_ctx_create(tt_ctx **out, const tt_grid *grid, void *cuda_stream) {
    if (!out || !grid) return TT_EINVAL;
    *out = nullptr;
    const tt_grid &G = *grid;
    GridC gc;
    if (!grid_constants(G, gc)) return TT_EINVAL;
    tt_ctx *ctx = new tt_ctx();
    ctx->grid = G;
    ctx->st = (cudaStream_t)cuda_stream;
    ctx->g = gc;
    tt_status s = TT_OK;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device) !=
            cudaSuccess)
        s = fail(ctx, TT_ECUDA, "no CUDA device");
    if (s == TT_OK) s = build_schedule(ctx, ctx->interior, 1);
    if (s == TT_OK) s = build_schedule(ctx, ctx->full, 0);
    for (int q = 0; q < kNumTileShapes && s == TT_OK; ++q)
        s = build_tile_schedule(ctx, ctx->tiled[q], kTileShapes[q]);
    if (s == TT_OK) s = upload_geo<float>(ctx, ctx->gf);
    if (s == TT_OK) s = upload_geo<double>(ctx, ctx->gd);
    for (int q = 0; q < 2 && s == TT_OK; ++q)
        if (cudaEventCreate(&ctx->ev_start[q]) != cudaSuccess ||
            cudaEventCreate(&ctx->ev_stop[q]) != cudaSuccess ||
            cudaEventCreate(&ctx->ev_net[q]) != cudaSuccess ||
            cudaEventCreate(&ctx->ev_kacc[q]) != cudaSuccess)
            s = fail(ctx, TT_ECUDA, "cudaEventCreate failed");
    if (s == TT_OK && cudaMallocHost((void **)&ctx->h_pinned, pinned_bytes()) != cudaSuccess)
        s = fail(ctx, TT_ENOMEM, "pinned host allocation failed");
    if (s != TT_OK) {
        tt_ctx_destroy(ctx);
        return s;
    }
    *out = ctx;
    return TT_OK;
}

void tt_ctx_destroy(tt_ctx *ctx) {
    if (!ctx) return;
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    else cudaDeviceSynchronize();
    Schedule *ss[] = {&ctx->interior, &ctx->full};
    for (Schedule *S : ss) {
        if (S->nodes) cudaFree(S->nodes);
        if (S->off) cudaFree(S->off);
    }
    for (TileSchedule &S : ctx->tiled) {
        if (S.tiles) cudaFree(S.tiles);
        if (S.off) cudaFree(S.off);
    }
    free_geo(ctx->gf);
    free_geo(ctx->gd);
    DevBuf *bufs[] = {&ctx->src, &ctx->pts, &ctx->rpts, &ctx->tabT, &ctx->tabP, &ctx->rec, &ctx->partial,
                      &ctx->conv, &ctx->iters, &ctx->nact, &ctx->bar, &ctx->flags, &ctx->cq,
                      &ctx->wq, &ctx->sidx, &ctx->next, &ctx->heads, &ctx->nheads, &ctx->JS,
                      &ctx->coef, &ctx->t0c, &ctx->net_theta, &ctx->net_x, &ctx->net_a,
                      &ctx->net_b, &ctx->net_y, &ctx->net_d1, &ctx->net_d2, &ctx->net_dy,
                      &ctx->net_wt, &ctx->net_part, &ctx->net_scr, &ctx->tune_tau, &ctx->tau_w,
                      &ctx->slot_srcc, &ctx->slot_int,
                      &ctx->net_wbf, &ctx->mg_tab, &ctx->mg_scr, &ctx->upd_part,
                      &ctx->tele_tau, &ctx->tele_aux, &ctx->net_img, &ctx->net_timg,
                      &ctx->net_rows, &ctx->ord_perm, &ctx->ord_pts, &ctx->ord_src,
                      &ctx->ord_tabT, &ctx->ord_tabP, &ctx->ord_tau, &ctx->ord_iters,
                      &ctx->ord_conv};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (ctx->h_loss) cudaFreeHost(ctx->h_loss);
    for (int q = 0; q < 2; ++q) {
        if (ctx->ev_start[q]) cudaEventDestroy(ctx->ev_start[q]);
        if (ctx->ev_stop[q]) cudaEventDestroy(ctx->ev_stop[q]);
        if (ctx->ev_net[q]) cudaEventDestroy(ctx->ev_net[q]);
        if (ctx->ev_kacc[q]) cudaEventDestroy(ctx->ev_kacc[q]);
    }
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->h_pts) cudaFreeHost(ctx->h_pts);
    delete ctx;
}

tt_status tt_forward(tt_ctx *ctx, const tt_model *model, const tt_point *h_src, int n_src,
                     void *d_tau, void *d_T, const tt_opts *opts, int *h_iters) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if ((s = check_sources(ctx, h_src, n_src)) != TT_OK) return s;
    if ((s = check_opts(ctx, opts)) != TT_OK) return s;
    if (!d_tau) return fail(ctx, TT_EINVAL, "tau must be non-NULL");
    if (model->dtype == TT_F32)
        return forward_impl<float>(ctx, model, h_src, n_src, d_tau, d_T, opts, h_iters);
    return forward_impl<double>(ctx, model, h_src, n_src, d_tau, d_T, opts, h_iters);
}

tt_status tt_misfit(tt_ctx *ctx, const void *d_T, int dtype, const tt_data *d, double *d_Tr,
                    double *d_chi, double *d_R) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_data(ctx, d)) != TT_OK) return s;
    if (!d_T || !d_R) return fail(ctx, TT_EINVAL, "tt_misfit: NULL argument");
    if (dtype != TT_F32 && dtype != TT_F64) return fail(ctx, TT_EINVAL, "bad dtype %d", dtype);
    const int S = 8 * d->n_rec;
    ENSURE(ctx->flags, kFlagInts * sizeof(int));
    ENSURE(ctx->rpts, sizeof(PointD) * (size_t)d->n_rec);
    ENSURE(ctx->cq, sizeof(long long) * S);
    ENSURE(ctx->wq, sizeof(double) * S);
    int *flags = (int *)ctx->flags.p;
    CK(cudaMemsetAsync(flags, 0, 4 * sizeof(int), ctx->st));
    if ((s = stage_to(ctx, d->h_rec, d->n_rec, (PointD *)ctx->rpts.p)) != TT_OK) return s;
    if ((s = enq_receivers(ctx, (const PointD *)ctx->rpts.p, d->n_rec, (long long *)ctx->cq.p,
                           (double *)ctx->wq.p, flags)) != TT_OK)
        return s;
    if ((s = enq_misfit(ctx, d_T, dtype, d, (const long long *)ctx->cq.p,
                        (const double *)ctx->wq.p, flags, d_Tr, d_chi, d_R)) != TT_OK)
        return s;
    Readback r = readback_view(ctx);
    CK(cudaMemcpyAsync(r.flags, flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (r.flags[1]) return fail(ctx, TT_EINVAL, "tt_misfit: receiver index out of range in the data");
    if (r.flags[2]) return fail(ctx, TT_EINVAL, "tt_misfit: receiver outside the grid");
    return TT_OK;
}

tt_status tt_adjoint(tt_ctx *ctx, const tt_model *model, const tt_point *h_src, int n_src,
                     const void *d_T, int n_rec, const tt_point *h_rec, const double *d_R,
                     void *d_P, const tt_opts *opts, int *h_iters) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if ((s = check_sources(ctx, h_src, n_src)) != TT_OK) return s;
    if ((s = check_opts(ctx, opts)) != TT_OK) return s;
    if (!d_T || !d_R || !d_P) return fail(ctx, TT_EINVAL, "tt_adjoint: NULL field");
    if (n_rec < 1 || !h_rec) return fail(ctx, TT_EINVAL, "need at least one receiver");
    for (int q = 0; q < n_rec; ++q)
        if (!inside(ctx, h_rec[q]))
            return fail(ctx, TT_EINVAL, "receiver %d (%g km, %g, %g) outside the grid", q,
                        h_rec[q].depth_km, h_rec[q].lat_deg, h_rec[q].lon_deg);
    if (model->dtype == TT_F32)
        return adjoint_impl<float>(ctx, model, h_src, n_src, d_T, n_rec, h_rec, d_R, d_P, opts,
                                   h_iters);
    return adjoint_impl<double>(ctx, model, h_src, n_src, d_T, n_rec, h_rec, d_R, d_P, opts,
                                h_iters);
}

tt_status tt_kernel(tt_ctx *ctx, const tt_model *model, int n_src, const void *d_T,
                    const void *d_P, double *d_Ks, double *d_Kxi, double *d_Keta) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if (n_src < 1 || n_src > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "n_src = %d outside 1..%d", n_src, TT_MAX_BATCH);
    if (!d_T || !d_P || !d_Ks || !d_Kxi || !d_Keta)
        return fail(ctx, TT_EINVAL, "tt_kernel: NULL argument");
    return enq_kernel(ctx, model, n_src, d_T, d_P, d_Ks, d_Kxi, d_Keta);
}

tt_status tt_misfit_cr(tt_ctx *ctx, const tt_cr_data *d, const double *d_Tr, double *d_chi_cr,
                       double *d_R) {
    if (!ctx) return TT_EINVAL;
    if (!d || !d->d_off || !d_Tr || !d_chi_cr || !d_R)
        return fail(ctx, TT_EINVAL, "tt_misfit_cr: NULL argument");
    if (d->n_src < 1 || d->n_src > TT_MAX_BATCH || d->n_rec < 1)
        return fail(ctx, TT_EINVAL, "tt_misfit_cr: n_src %d or n_rec %d out of range", d->n_src,
                    d->n_rec);
    if (d->n_entries > 0 && (!d->d_other || !d->d_dtobs || !d->d_w))
        return fail(ctx, TT_EINVAL, "tt_misfit_cr: NULL entry arrays");
    ENSURE(ctx->flags, kFlagInts * sizeof(int));
    int *bad = (int *)ctx->flags.p + 1;
    CK(cudaMemsetAsync(bad, 0, sizeof(int), ctx->st));
    CK(run_misfit_cr(d->n_src, d->n_rec, d->d_off, d->d_other, d->d_dtobs, d->d_w, d->gamma, d_Tr,
                     d_chi_cr, d_R, bad, ctx->st));
    ctx->launches += 1;
    int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h_bad) return fail(ctx, TT_EINVAL, "tt_misfit_cr: an entry names a source out of range");
    return TT_OK;
}

tt_status tt_cr_pack(tt_ctx *ctx, int n_src, int n_rec, int n_pairs, const double *h_pairs,
                     int *h_off, int *h_other, double *h_dtobs, double *h_w) {
    if (n_src < 1 || n_src > TT_MAX_BATCH || n_rec < 1 || n_pairs < 0)
        return fail(ctx, TT_EINVAL, "tt_cr_pack: n_src %d, n_rec %d or n_pairs %d out of range",
                    n_src, n_rec, n_pairs);
    if (!h_off || (n_pairs > 0 && (!h_pairs || !h_other || !h_dtobs || !h_w)))
        return fail(ctx, TT_EINVAL, "tt_cr_pack: NULL argument");
    if ((long long)n_src * n_rec + 1 > 0x7fffffffLL || 2LL * n_pairs > 0x7fffffffLL)
        return fail(ctx, TT_EINVAL, "tt_cr_pack: table too large for int offsets");
    // source, other source and receiver of every pair, checked before anything is written
    for (int p = 0; p < n_pairs; ++p) {
        const double *e = h_pairs + 5LL * p;
        const double b = e[0], j = e[1], m = e[2];
        if (!(b >= 0 && b < n_src && b == (double)(int)b) ||
            !(j >= 0 && j < n_src && j == (double)(int)j) ||
            !(m >= 0 && m < n_rec && m == (double)(int)m) || b == j)
            return fail(ctx, TT_EINVAL,
                        "tt_cr_pack: pair %d (%g, %g, %g) is not two distinct sources below %d "
                        "at a receiver below %d",
                        p, b, j, m, n_src, n_rec);
    }
    // Counting sort by (source, receiver). The pairs are listed first under their first
    // source with dT_obs, then under their second with -dT_obs, each in the order given;
    // that order is kept among the entries of one (source, receiver).
    const long long n_keys = (long long)n_src * n_rec;
    for (long long q = 0; q <= n_keys; ++q) h_off[q] = 0;
    for (int p = 0; p < n_pairs; ++p) {
        const double *e = h_pairs + 5LL * p;
        const int m = (int)e[2];
        h_off[(long long)(int)e[0] * n_rec + m + 1] += 1;
        h_off[(long long)(int)e[1] * n_rec + m + 1] += 1;
    }
    for (long long q = 0; q < n_keys; ++q) h_off[q + 1] += h_off[q];
    std::vector<int> next(h_off, h_off + n_keys);
    for (int pass = 0; pass < 2; ++pass)
        for (int p = 0; p < n_pairs; ++p) {
            const double *e = h_pairs + 5LL * p;
            const int src = (int)e[pass], oth = (int)e[1 - pass], m = (int)e[2];
            const int q = next[(long long)src * n_rec + m]++;
            h_other[q] = oth;
            h_dtobs[q] = pass == 0 ? e[3] : -e[3];
            h_w[q] = e[4];
        }
    return TT_OK;
}

tt_status tt_kernel_density(tt_ctx *ctx, const void *d_P, int n_src, int dtype, double *d_Kd) {
    if (!ctx) return TT_EINVAL;
    if (n_src < 1 || n_src > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "n_src = %d outside 1..%d", n_src, TT_MAX_BATCH);
    if (dtype != TT_F32 && dtype != TT_F64)
        return fail(ctx, TT_EINVAL, "dtype %d is neither TT_F32 nor TT_F64", dtype);
    if (!d_P || !d_Kd) return fail(ctx, TT_EINVAL, "tt_kernel_density: NULL argument");
    const long long N = ctx->g.N;
    CK(dtype == TT_F32 ? run_kernel_density<float>(N, n_src, (const float *)d_P, d_Kd, ctx->st)
                       : run_kernel_density<double>(N, n_src, (const double *)d_P, d_Kd, ctx->st));
    ctx->launches += 1;
    return TT_OK;
}

tt_status tt_field_at_points(tt_ctx *ctx, const void *d_G, int dtype, int n_fields, int n_pts,
                             const double *d_pts, double *d_val, double *d_grad) {
    if (!ctx) return TT_EINVAL;
    if (!d_G || !d_pts || !d_val || !d_grad)
        return fail(ctx, TT_EINVAL, "tt_field_at_points: NULL argument");
    if (dtype != TT_F32 && dtype != TT_F64)
        return fail(ctx, TT_EINVAL, "dtype %d is neither TT_F32 nor TT_F64", dtype);
    if (n_fields < 1 || n_fields > TT_MAX_BATCH || n_pts < 1 || n_pts > (1 << 24))
        return fail(ctx, TT_EINVAL, "tt_field_at_points: n_fields %d or n_pts %d out of range",
                    n_fields, n_pts);
    ENSURE(ctx->flags, kFlagInts * sizeof(int));
    int *bad = (int *)ctx->flags.p + 1;
    CK(cudaMemsetAsync(bad, 0, sizeof(int), ctx->st));
    CK(dtype == TT_F32 ? run_field_at_points<float>(ctx->g, n_fields, n_pts, d_G, d_pts, d_val,
                                                    d_grad, bad, ctx->st)
                       : run_field_at_points<double>(ctx->g, n_fields, n_pts, d_G, d_pts, d_val,
                                                     d_grad, bad, ctx->st));
    ctx->launches += 1;
    int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h_bad) return fail(ctx, TT_EINVAL, "tt_field_at_points: a point lies outside the grid");
    return TT_OK;
}

tt_status tt_misfit_table(tt_ctx *ctx, const double *d_val, const double *d_otime,
                          const tt_data *d, double *d_Tr, double *d_chi, double *d_R) {
    if (!ctx) return TT_EINVAL;
    if (!d || !d->d_abs_off || !d->d_cs_off || !d_val || !d_R)
        return fail(ctx, TT_EINVAL, "tt_misfit_table: NULL argument");
    if (d->n_src < 1 || d->n_src > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "n_src = %d outside 1..%d", d->n_src, TT_MAX_BATCH);
    if (d->n_rec < 1) return fail(ctx, TT_EINVAL, "need at least one receiver");
    if ((size_t)d->n_rec * 2 * 4 * sizeof(double) > 200 * 1024)
        return fail(ctx, TT_EINVAL, "n_rec = %d too large for the misfit kernel", d->n_rec);
    ENSURE(ctx->flags, kFlagInts * sizeof(int));
    int *bad = (int *)ctx->flags.p + 1;
    CK(cudaMemsetAsync(bad, 0, sizeof(int), ctx->st));
    CK(run_misfit_table(d->n_src, d->n_rec, d_val, d_otime, *d, d_Tr, d_chi, d_R, bad, ctx->st));
    ctx->launches += 1;
    int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h_bad) return fail(ctx, TT_EINVAL, "tt_misfit_table: receiver index out of range in the data");
    return TT_OK;
}

tt_status tt_reloc_kernels(tt_ctx *ctx, int n_src, int n_rec, const double *d_R,
                           const double *d_grad, double *d_Kx, double *d_Ktau) {
    if (!ctx) return TT_EINVAL;
    if (!d_R || !d_grad || !d_Kx || !d_Ktau)
        return fail(ctx, TT_EINVAL, "tt_reloc_kernels: NULL argument");
    if (n_src < 1 || n_src > (1 << 24) || n_rec < 1 || n_rec > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "tt_reloc_kernels: n_src %d or n_rec %d out of range", n_src,
                    n_rec);
    CK(run_reloc_kernels(n_src, n_rec, d_R, d_grad, d_Kx, d_Ktau, ctx->st));
    ctx->launches += 1;
    return TT_OK;
}

tt_status tt_reloc_update(tt_ctx *ctx, int n_src, double *d_pts, double *d_otime,
                          const double *d_Kx, const double *d_Ktau, double step_km,
                          double step_s) {
    if (!ctx) return TT_EINVAL;
    if (!d_pts || !d_Kx || !d_Ktau) return fail(ctx, TT_EINVAL, "tt_reloc_update: NULL argument");
    if (n_src < 1 || n_src > (1 << 24))
        return fail(ctx, TT_EINVAL, "tt_reloc_update: n_src %d out of range", n_src);
    if (!(step_km >= 0.0 && step_km < 1e300) || !(step_s >= 0.0 && step_s < 1e300))
        return fail(ctx, TT_EINVAL, "tt_reloc_update: steps must be finite and >= 0");
    const tt_grid &gr = ctx->grid;
    const GridBox box{{gr.depth_min_km, gr.lat_min_deg, gr.lon_min_deg},
                      {gr.depth_max_km, gr.lat_max_deg, gr.lon_max_deg}};
    CK(run_reloc_update(ctx->g, box, n_src, d_pts, d_otime, d_Kx, d_Ktau, step_km, step_s,
                        ctx->st));
    ctx->launches += 1;
    return TT_OK;
}

tt_status tt_tele2d(tt_ctx *ctx, int dtype, int n_r, int n_d, double r_min_km, double r_max_km,
                    double d_max_deg, const void *d_s_r, int n_ev, const double *h_r_src_km,
                    double tol, int max_iter, void *d_T, int *h_iters) {
    if (!ctx) return TT_EINVAL;
    if (dtype != TT_F32 && dtype != TT_F64)
        return fail(ctx, TT_EINVAL, "dtype %d is neither TT_F32 nor TT_F64", dtype);
    if (!d_s_r || !h_r_src_km || !d_T) return fail(ctx, TT_EINVAL, "tt_tele2d: NULL argument");
    if (n_r < 4 || n_d < 4 || n_r > 1 << 14 || n_d > 1 << 14 || n_ev < 1 || n_ev > 1 << 16)
        return fail(ctx, TT_EINVAL, "tt_tele2d: n_r %d, n_d %d (4..16384) or n_ev %d out of range",
                    n_r, n_d, n_ev);
    if (!(r_max_km > r_min_km) || !(r_min_km > 0.0) || !(d_max_deg > 0.0 && d_max_deg <= 180.0))
        return fail(ctx, TT_EINVAL, "tt_tele2d: bad 2-D grid extent");
    if (!(tol > 0.0) || max_iter < 1) return fail(ctx, TT_EINVAL, "tt_tele2d: bad tol or max_iter");
    for (int e = 0; e < n_ev; ++e)
        if (!(h_r_src_km[e] >= r_min_km && h_r_src_km[e] <= r_max_km))
            return fail(ctx, TT_EINVAL, "tt_tele2d: event %d at radius %g outside the 2-D grid", e,
                        h_r_src_km[e]);
    const size_t fs = dtype == TT_F32 ? sizeof(float) : sizeof(double);
    ENSURE(ctx->tele_tau, fs * (size_t)n_ev * n_r * n_d);
    ENSURE(ctx->tele_aux, sizeof(double) * (size_t)n_ev + sizeof(int) * (size_t)n_ev);
    double *d_rs = (double *)ctx->tele_aux.p;
    int *d_it = (int *)(d_rs + n_ev);
    CK(cudaMemcpyAsync(d_rs, h_r_src_km, sizeof(double) * n_ev, cudaMemcpyHostToDevice, ctx->st));
    const double dr = (r_max_km - r_min_km) / (n_r - 1);
    const double dd = d_max_deg * (3.14159265358979323846 / 180.0) / (n_d - 1);
    CK(dtype == TT_F32 ? run_tele2d<float>(n_r, n_d, r_min_km, dr, dd, d_s_r, d_rs, n_ev, tol,
                                           max_iter, ctx->tele_tau.p, d_T, d_it, ctx->st)
                       : run_tele2d<double>(n_r, n_d, r_min_km, dr, dd, d_s_r, d_rs, n_ev, tol,
                                            max_iter, ctx->tele_tau.p, d_T, d_it, ctx->st));
    ctx->launches += 1;
    std::vector<int> it(n_ev);
    CK(cudaMemcpyAsync(it.data(), d_it, sizeof(int) * n_ev, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    int bad = 0;
    for (int e = 0; e < n_ev; ++e) {
        if (h_iters) h_iters[e] = it[e];
        bad += it[e] >= max_iter;
    }
    if (bad)
        return fail(ctx, TT_ENOTCONVERGED, "tt_tele2d: %d of %d events did not converge in %d iterations",
                    bad, n_ev, max_iter);
    return TT_OK;
}

tt_status tt_tele_region_times(tt_ctx *ctx, int dtype, int n_r, int n_d, double r_min_km,
                               double r_max_km, double d_max_deg, const void *d_T2, int n_ev,
                               const tt_point *h_events, void *d_T) {
    if (!ctx) return TT_EINVAL;
    if (dtype != TT_F32 && dtype != TT_F64)
        return fail(ctx, TT_EINVAL, "dtype %d is neither TT_F32 nor TT_F64", dtype);
    if (!d_T2 || !h_events || !d_T) return fail(ctx, TT_EINVAL, "tt_tele_region_times: NULL argument");
    if (n_r < 4 || n_d < 4 || n_ev < 1 || n_ev > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "tt_tele_region_times: sizes out of range");
    const tt_grid &gr = ctx->grid;
    const double deg = 3.14159265358979323846 / 180.0;
    const double r_lo = gr.earth_radius_km - gr.depth_max_km, r_hi = gr.earth_radius_km - gr.depth_min_km;
    if (gr.geometry != 0 || r_lo < r_min_km - 1e-9 || r_hi > r_max_km + 1e-9)
        return fail(ctx, TT_EINVAL, "tt_tele_region_times: the 2-D radii do not cover the spherical region");
    std::vector<double> ll(2 * (size_t)n_ev);
    for (int e = 0; e < n_ev; ++e) {
        ll[2 * e] = h_events[e].lat_deg * deg;
        ll[2 * e + 1] = h_events[e].lon_deg * deg;
        // the region's largest epicentral angle: its eight corners bound it on a small region
        for (int c = 0; c < 4; ++c) {
            const double th = (c & 1 ? gr.lat_max_deg : gr.lat_min_deg) * deg;
            const double ph = (c & 2 ? gr.lon_max_deg : gr.lon_min_deg) * deg;
            double cd = sin(th) * sin(ll[2 * e]) + cos(th) * cos(ll[2 * e]) * cos(ph - ll[2 * e + 1]);
            cd = cd > 1.0 ? 1.0 : (cd < -1.0 ? -1.0 : cd);
            if (acos(cd) > d_max_deg * deg)
                return fail(ctx, TT_EINVAL, "tt_tele_region_times: event %d is farther than the 2-D grid's %g deg", e, d_max_deg);
        }
    }
    ENSURE(ctx->tele_aux, sizeof(double) * 2 * (size_t)n_ev);
    CK(cudaMemcpyAsync(ctx->tele_aux.p, ll.data(), sizeof(double) * 2 * n_ev, cudaMemcpyHostToDevice,
                       ctx->st));
    const double dr2 = (r_max_km - r_min_km) / (n_r - 1);
    const double dd = d_max_deg * deg / (n_d - 1);
    CK(dtype == TT_F32 ? run_region_times<float>(ctx->g, n_r, n_d, r_min_km, dr2, dd, d_T2, n_ev,
                                                 (const double *)ctx->tele_aux.p, d_T, ctx->st)
                       : run_region_times<double>(ctx->g, n_r, n_d, r_min_km, dr2, dd, d_T2, n_ev,
                                                  (const double *)ctx->tele_aux.p, d_T, ctx->st));
    ctx->launches += 1;
    CK(cudaStreamSynchronize(ctx->st));
    return TT_OK;
}

}  // extern "C"

namespace {

// The region's solve of teleseismic events (R17): one persistent cooperative launch of the
// node-hyperplane sweep with SCHEME 3 (Lax-Friedrichs on T itself, faces held fixed), the
// events as the batch, each stopping on its own criterion inside the launch.
template <typename F>
tt_status forward_tele_impl(tt_ctx *ctx, const tt_model *m, int n_ev, void *d_T,
                            const tt_opts *o, int *h_iters) {
    const GridC &g = ctx->g;
    ENSURE(ctx->rec, sizeof(NodeRec<F>) * (size_t)g.N);
    ENSURE(ctx->partial, partial_bytes(ctx, n_ev, sizeof(F)));
    ENSURE(ctx->conv, sizeof(int) * (size_t)n_ev);
    ENSURE(ctx->iters, sizeof(int) * (size_t)n_ev);
    ENSURE(ctx->nact, sizeof(int) * kMaxBarrierGroups);
    ENSURE(ctx->bar, sizeof(BarrierState) * kMaxBarrierGroups);
    ENSURE(ctx->flags, kFlagInts * sizeof(int));
    NodeRec<F> *rec = (NodeRec<F> *)ctx->rec.p;
    int *conv = (int *)ctx->conv.p, *iters = (int *)ctx->iters.p, *flags = (int *)ctx->flags.p;
    BarrierState *bar = (BarrierState *)ctx->bar.p;
    CK(cudaMemsetAsync(conv, 0, sizeof(int) * (size_t)n_ev, ctx->st));
    CK(cudaMemsetAsync(iters, 0, sizeof(int) * (size_t)n_ev, ctx->st));
    CK(cudaMemsetAsync(ctx->nact.p, 0, sizeof(int) * kMaxBarrierGroups, ctx->st));
    CK(cudaMemsetAsync(bar, 0, sizeof(BarrierState) * kMaxBarrierGroups, ctx->st));
    CK(cudaMemsetAsync(flags, 0, 4 * sizeof(int), ctx->st));
    CK(run_node_records<F>(g, m->d_s, m->d_xi, m->d_eta, ctx->gd.h2, ctx->gd.cost, rec, flags,
                           ctx->st));
    ENSURE(ctx->tele_aux, sizeof(F) * (size_t)n_ev);
    CK(run_tele_shift<F>(g.N, n_ev, d_T, ctx->tele_aux.p, -1, ctx->st));
    FwdArgs<F> a;
    memset(&a, 0, sizeof a);
    a.g = g;
    a.B = n_ev;
    a.scheme = 3;
    a.n_planes = ctx->interior.n_planes;
    a.er = (F)(0.5 / g.dr);
    a.rec = rec;
    a.tau = (F *)d_T;
    a.nodes = ctx->interior.nodes;
    a.off = ctx->interior.off;
    a.bar = bar;
    a.partial = (F *)ctx->partial.p;
    a.conv = conv;
    a.iters = iters;
    a.n_active = (int *)ctx->nact.p;
    a.tol = (F)o->tol_fwd;
    a.max_iter = o->max_iter_fwd;
    a.spin_ns = spin_ns(o);
    a.src_lo = 0;
    a.src_n = n_ev;
    a.idx32 = (unsigned long long)g.N * (unsigned long long)(n_ev > 8 ? n_ev : 8) < (1ull << 32);
    // 256-thread blocks, one barrier group per resident block slot of an SM (as the
    // forward sweep), each group a multiple of one warp's sources
    const int block = 256;
    int per_sm = forward_blocks_per_sm<F>(block, fwd_smem_bytes<F>(n_ev, block), a.idx32 != 0, 3);
    if (per_sm <= 0) return fail(ctx, TT_ECUDA, "teleseismic sweep cannot be resident");
    if (per_sm > kMaxBarrierGroups) per_sm = kMaxBarrierGroups;
    int max_grid = per_sm * ctx->n_sm;
    if (o->launch_blocks > 0 && o->launch_blocks < max_grid) max_grid = o->launch_blocks;
    const int wsrc = 32 * kFwdSourcesPerLane;
    int groups = o->fwd_groups > 0 ? o->fwd_groups : per_sm;
    if (groups > (n_ev + wsrc - 1) / wsrc) groups = (n_ev + wsrc - 1) / wsrc;
    if (groups > max_grid) groups = max_grid;
    int gsrc = ((n_ev + groups - 1) / groups + wsrc - 1) / wsrc * wsrc;
    groups = (n_ev + gsrc - 1) / gsrc;
    int gblocks = max_grid / groups;
    if ((long long)gblocks * block < gsrc) {
        const int need = (gsrc + block - 1) / block;
        if ((long long)need * groups > (long long)per_sm * ctx->n_sm)
            return fail(ctx, TT_EINVAL, "%d events exceed one resident launch", n_ev);
        gblocks = need;
    }
    a.n_bgroups = groups;
    a.grp_blocks = gblocks;
    a.grp_src = gsrc;
    CK(record(ctx, ctx->ev_start[TT_STATS_FORWARD]));
    CK(launch_forward<F>(a, gblocks * groups, block, ctx->st));
    CK(record(ctx, ctx->ev_stop[TT_STATS_FORWARD]));
    CK(run_tele_shift<F>(g.N, n_ev, d_T, ctx->tele_aux.p, 1, ctx->st));
    ctx->launches += 5;
    Readback r = readback_view(ctx);
    CK(cudaMemcpyAsync(r.iters_f, iters, sizeof(int) * (size_t)n_ev, cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaMemcpyAsync(r.conv_f, conv, sizeof(int) * (size_t)n_ev, cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaMemcpyAsync(r.flags, flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(r.bar_f, bar, sizeof(BarrierState) * kMaxBarrierGroups,
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (r.flags[0] & 1)
        return fail(ctx, TT_EINVAL, "tt_forward_tele: model has s <= 0 or xi^2 + eta^2 >= 1/4");
    for (int q = 0; q < kMaxBarrierGroups; ++q) {
        int st;
        memcpy(&st, r.bar_f + q * sizeof(BarrierState) + offsetof(BarrierState, status),
               sizeof st);
        if (st == kDevTimeout)
            return fail(ctx, TT_ETIMEOUT, "tt_forward_tele: a device-side wait exceeded its limit");
    }
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev_start[TT_STATS_FORWARD], ctx->ev_stop[TT_STATS_FORWARD]));
    tt_stats &S = ctx->stats[TT_STATS_FORWARD];
    S = tt_stats{};
    S.sweep_ms = ms;
    long long upd = 0;
    int imax = 0, left = 0;
    const long long inner = (long long)(g.nr - 2) * (g.nt - 2) * (g.np - 2);
    for (int e = 0; e < n_ev; ++e) {
        upd += 8LL * r.iters_f[e] * inner;
        imax = r.iters_f[e] > imax ? r.iters_f[e] : imax;
        left += r.conv_f[e] == 0;
        if (h_iters) h_iters[e] = r.iters_f[e];
    }
    S.node_updates = upd;
    S.node_sweeps = 8LL * imax * inner;
    S.iters_max = imax;
    S.grid_blocks = gblocks * groups;
    S.block_threads = block;
    if (left)
        return fail(ctx, TT_ENOTCONVERGED,
                    "tt_forward_tele: %d of %d events did not converge in %d iterations", left,
                    n_ev, o->max_iter_fwd);
    return TT_OK;
}

}  // namespace

extern "C" {

tt_status tt_forward_tele(tt_ctx *ctx, const tt_model *model, int n_ev, void *d_T,
                          const tt_opts *opts, int *h_iters) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if ((s = check_opts(ctx, opts)) != TT_OK) return s;
    if (!d_T) return fail(ctx, TT_EINVAL, "tt_forward_tele: NULL field");
    if (n_ev < 1 || n_ev > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "n_ev = %d outside 1..%d", n_ev, TT_MAX_BATCH);
    return model->dtype == TT_F32 ? forward_tele_impl<float>(ctx, model, n_ev, d_T, opts, h_iters)
                                  : forward_tele_impl<double>(ctx, model, n_ev, d_T, opts, h_iters);
}

tt_status tt_kernel_normalize(tt_ctx *ctx, double *d_Ks, double *d_Kxi, double *d_Keta,
                              const double *d_Kd, double eps, double zeta) {
    if (!ctx) return TT_EINVAL;
    if (!d_Ks || !d_Kxi || !d_Keta || !d_Kd)
        return fail(ctx, TT_EINVAL, "tt_kernel_normalize: NULL argument");
    if (!(eps > 0) || !(zeta >= 0))
        return fail(ctx, TT_EINVAL, "tt_kernel_normalize: eps must be > 0 and zeta >= 0");
    CK(run_kernel_normalize(ctx->g.N, d_Ks, d_Kxi, d_Keta, d_Kd, eps, zeta, ctx->st));
    ctx->launches += 1;
    return TT_OK;
}

}  // extern "C"

namespace {

// The tables of the inversion grids of mg on the device, rebuilt when mg changes: Wr, Wt, Wp
// (double) then lo for r, theta, phi (int).
struct MgTabs {
    const double *Wr, *Wt, *Wp;
    const int *lo;
};

tt_status mgrid_tables(tt_ctx *ctx, const tt_mgrid *mg, MgDims &d, MgTabs &tb) {
    if (!mg) return fail(ctx, TT_EINVAL, "inversion grid description is NULL");
    if (mg->n_grids < 1 || mg->n_grids > 64 || mg->n_r < 3 || mg->n_t < 3 || mg->n_p < 3 ||
        mg->n_r > 4096 || mg->n_t > 4096 || mg->n_p > 4096)
        return fail(ctx, TT_EINVAL, "inversion grids: need 1..64 grids of 3..4096 nodes per axis");
    const GridC &g = ctx->g;
    d = MgDims{g.nr, g.nt, g.np, mg->n_r, mg->n_t, mg->n_p, mg->n_grids};
    const size_t nw = (size_t)d.H * ((size_t)d.cr * d.nr + (size_t)d.ct * d.nt + (size_t)d.cp * d.np);
    const size_t nl = (size_t)d.H * ((size_t)d.nr + d.nt + d.np);
    ENSURE(ctx->mg_tab, sizeof(double) * nw + sizeof(int) * nl);
    double *W = (double *)ctx->mg_tab.p;
    tb.Wr = W;
    tb.Wt = W + (size_t)d.H * d.cr * d.nr;
    tb.Wp = tb.Wt + (size_t)d.H * d.ct * d.nt;
    tb.lo = (const int *)(W + nw);
    const int key[4] = {mg->n_r, mg->n_t, mg->n_p, mg->n_grids};
    if (memcmp(key, ctx->mg_key, sizeof key) == 0) return TT_OK;
    std::vector<double> hw, w;
    std::vector<int> hl, l;
    const int n[3] = {d.nr, d.nt, d.np}, c[3] = {d.cr, d.ct, d.cp};
    for (int a = 0; a < 3; ++a) {
        mgrid_axis_tables(n[a], c[a], d.H, w, l);
        hw.insert(hw.end(), w.begin(), w.end());
        hl.insert(hl.end(), l.begin(), l.end());
    }
    CK(cudaStreamSynchronize(ctx->st));   // the previous tables may still be read
    CK(cudaMemcpy(W, hw.data(), sizeof(double) * nw, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(W + nw, hl.data(), sizeof(int) * nl, cudaMemcpyHostToDevice));
    memcpy(ctx->mg_key, key, sizeof key);
    return TT_OK;
}

}  // namespace

extern "C" {

tt_status tt_mgrid_project(tt_ctx *ctx, const tt_mgrid *mg, const double *d_K, double *d_G) {
    if (!ctx) return TT_EINVAL;
    if (!d_K || !d_G) return fail(ctx, TT_EINVAL, "tt_mgrid_project: NULL argument");
    MgDims d;
    MgTabs tb;
    tt_status s;
    if ((s = mgrid_tables(ctx, mg, d, tb)) != TT_OK) return s;
    const size_t n1 = (size_t)d.H * d.nr * d.nt * d.cp, n2 = (size_t)d.H * d.nr * d.ct * d.cp;
    ENSURE(ctx->mg_scr, sizeof(double) * (n1 + n2));
    double *T1 = (double *)ctx->mg_scr.p;
    const GridC &g = ctx->g;
    CK(run_mgrid_project(d, d_K, ctx->gd.h2, ctx->gd.cost, g.dr * g.dt * g.dp, tb.Wr, tb.Wt,
                         tb.Wp, T1, T1 + n1, d_G, ctx->st));
    ctx->launches += 3;
    return TT_OK;
}

tt_status tt_mgrid_expand(tt_ctx *ctx, const tt_mgrid *mg, const double *d_G, double *d_D) {
    if (!ctx) return TT_EINVAL;
    if (!d_G || !d_D) return fail(ctx, TT_EINVAL, "tt_mgrid_expand: NULL argument");
    MgDims d;
    MgTabs tb;
    tt_status s;
    if ((s = mgrid_tables(ctx, mg, d, tb)) != TT_OK) return s;
    CK(run_mgrid_expand(d, d_G, tb.lo, tb.Wr, tb.Wt, tb.Wp, d_D, ctx->st));
    ctx->launches += 1;
    return TT_OK;
}

tt_status tt_kernel_normalize_rel(tt_ctx *ctx, double *d_Ks, double *d_Kxi, double *d_Keta,
                                  const double *d_Kd, double eps_rel, double zeta) {
    if (!ctx) return TT_EINVAL;
    if (!d_Ks || !d_Kxi || !d_Keta || !d_Kd)
        return fail(ctx, TT_EINVAL, "tt_kernel_normalize_rel: NULL argument");
    if (!(eps_rel > 0) || !(zeta >= 0))
        return fail(ctx, TT_EINVAL, "tt_kernel_normalize_rel: eps_rel must be > 0 and zeta >= 0");
    constexpr int kParts = 304;
    ENSURE(ctx->upd_part, sizeof(double) * (3 * kParts + 3));
    CK(run_kernel_normalize_rel(ctx->g.N, d_Ks, d_Kxi, d_Keta, d_Kd, eps_rel, zeta,
                                (double *)ctx->upd_part.p, kParts, ctx->st));
    ctx->launches += 3;
    return TT_OK;
}

tt_status tt_misfit_total(tt_ctx *ctx, int n_src, const double *d_chi, double alpha, double beta,
                          const double *d_chi_cr, double gamma, double *h_total) {
    if (!ctx) return TT_EINVAL;
    if (!d_chi || !h_total || n_src < 1 || n_src > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "tt_misfit_total: NULL argument or n_src outside 1..%d",
                    TT_MAX_BATCH);
    ENSURE(ctx->upd_part, sizeof(double) * (3 * 304 + 3));
    double *d_out = (double *)ctx->upd_part.p;
    CK(run_misfit_total(n_src, d_chi, alpha, beta, d_chi_cr, gamma, d_out, ctx->st));
    ctx->launches += 1;
    double *h = pinned_scalar(ctx);
    CK(cudaMemcpyAsync(h, d_out, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *h_total = *h;
    return TT_OK;
}

tt_status tt_model_update(tt_ctx *ctx, const tt_model *model, const double *d_Ds,
                          const double *d_Dxi, const double *d_Deta, double step) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if (!d_Ds || !d_Dxi || !d_Deta) return fail(ctx, TT_EINVAL, "tt_model_update: NULL direction");
    if (!(step > 0) || !(step < 1)) return fail(ctx, TT_EINVAL, "tt_model_update: step must be in (0, 1)");
    constexpr int kParts = 304;   // 2 x 152 SMs
    ENSURE(ctx->upd_part, sizeof(double) * (3 * kParts + 3));
    double *part = (double *)ctx->upd_part.p;
    const long long N = ctx->g.N;
    if (model->dtype == TT_F32)
        CK(run_model_update<float>(N, (float *)model->d_s, (float *)model->d_xi,
                                   (float *)model->d_eta, d_Ds, d_Dxi, d_Deta, step, part, kParts,
                                   ctx->st));
    else
        CK(run_model_update<double>(N, (double *)model->d_s, (double *)model->d_xi,
                                    (double *)model->d_eta, d_Ds, d_Dxi, d_Deta, step, part,
                                    kParts, ctx->st));
    ctx->launches += 3;
    return TT_OK;
}

tt_status tt_get_stats(const tt_ctx *ctx, int which, tt_stats *out) {
    if (!ctx || !out ||
        (which != TT_STATS_FORWARD && which != TT_STATS_ADJOINT && which != TT_STATS_KERNEL))
        return TT_EINVAL;
    if (which == TT_STATS_KERNEL) {
        // the last kernel accumulation: waits for it, then reads its events
        tt_stats S = {};
        if (ctx->kacc_B > 0) {
            float ms = 0.f;
            if (cudaEventSynchronize(ctx->ev_kacc[1]) != cudaSuccess ||
                cudaEventElapsedTime(&ms, ctx->ev_kacc[0], ctx->ev_kacc[1]) != cudaSuccess)
                return TT_ECUDA;
            S.sweep_ms = ms;
            S.node_updates = ctx->g.N * (long long)ctx->kacc_B;
            S.node_sweeps = ctx->g.N;
            S.iters_max = 1;
        }
        *out = S;
        out->launches = ctx->launches;
        return TT_OK;
    }
    *out = ctx->stats[which];
    out->launches = ctx->launches;
    return TT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- autotuner

namespace {

constexpr int kTuneCandidates = 7;

template <typename F>
tt_status autotune_impl(tt_ctx *ctx, const tt_model *m, const tt_point *h_src, int B,
                        tt_opts *opts, double *h_ms) {
    tt_status s;
    ENSURE(ctx->tune_tau, sizeof(F) * (size_t)ctx->g.N * B);
    const bool tiles_ok = B >= 32 && (B * sizeof(F)) % 16 == 0;
    double best = 1e300;
    int best_sched = 1, best_groups = 0;
    std::vector<int> it(B);
    for (int c = 0; c < kTuneCandidates; ++c) {
        tt_opts o = *opts;
        o.init = 0;
        // Lax-Friedrichs: two iterations show the per-iteration cost. The Godunov solvers
        // converge in a handful of iterations, and the sources' unequal counts decide how
        // barrier groups share the GPU, so they run the whole solve (node hyperplanes only).
        if (opts->scheme == 0) o.max_iter_fwd = 2;
        o.sweep_schedule = c < 4 ? 1 : c - 2;
        o.fwd_groups = c < 4 ? (1 << c) : 0;
        double ms = 0.0;
        if (c < 4 || (tiles_ok && opts->scheme == 0)) {
            s = forward_impl<F>(ctx, m, h_src, B, ctx->tune_tau.p, nullptr, &o, it.data());
            if (s != TT_OK && s != TT_ENOTCONVERGED) return s;
            int imax = 0;
            for (int b = 0; b < B; ++b) imax = it[b] > imax ? it[b] : imax;
            ms = ctx->stats[TT_STATS_FORWARD].sweep_ms / (imax > 0 ? imax : 1);
            if (ms < best) {
                best = ms;
                best_sched = o.sweep_schedule;
                best_groups = o.fwd_groups;
            }
        }
        if (h_ms) h_ms[c] = ms;
    }
    ctx->tuned.push_back({B, m->dtype, opts->scheme, best_sched, best_groups});
    opts->sweep_schedule = best_sched;
    opts->fwd_groups = best_groups;
    return TT_OK;
}

}  // namespace

extern "C" tt_status tt_autotune(tt_ctx *ctx, const tt_model *model, const tt_point *h_src,
                                 int n_src, tt_opts *opts, double *h_ms) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if ((s = check_sources(ctx, h_src, n_src)) != TT_OK) return s;
    if ((s = check_opts(ctx, opts)) != TT_OK) return s;
    for (const auto &t : ctx->tuned)
        if (t.n_src == n_src && t.dtype == model->dtype && t.scheme == opts->scheme) {
            opts->sweep_schedule = t.schedule;
            opts->fwd_groups = t.groups;
            if (h_ms)
                for (int c = 0; c < kTuneCandidates; ++c) h_ms[c] = 0.0;
            return TT_OK;
        }
    return model->dtype == TT_F32 ? autotune_impl<float>(ctx, model, h_src, n_src, opts, h_ms)
                                  : autotune_impl<double>(ctx, model, h_src, n_src, opts, h_ms);
}

// Adjoint launch configurations timed by tt_autotune_adjoint: (adj_chunk, adj_groups).
constexpr int kAdjTuneCandidates = 6;
constexpr int kAdjTuneChunk[kAdjTuneCandidates] = {0, 0, 0, 0, 128, 64};
constexpr int kAdjTuneGroups[kAdjTuneCandidates] = {1, 2, 4, 8, 0, 1};

namespace {

template <typename F>
tt_status autotune_adjoint_impl(tt_ctx *ctx, const tt_model *m, const tt_point *h_src, int B,
                                const void *d_T, int n_rec, const tt_point *h_rec,
                                const double *d_R, tt_opts *opts, double *h_ms) {
    tt_status s;
    ENSURE(ctx->tune_tau, sizeof(F) * (size_t)ctx->g.N * B);
    double best = 1e300;
    int best_c = 0;
    std::vector<int> it(B);
    for (int c = 0; c < kAdjTuneCandidates; ++c) {
        tt_opts o = *opts;
        o.adj_chunk = kAdjTuneChunk[c];
        o.adj_groups = kAdjTuneGroups[c];
        double ms = 0.0;
        // a chunk no smaller than the batch repeats an all-sources candidate
        const bool distinct = o.adj_chunk == 0 || o.adj_chunk < B;
        if (distinct && (o.adj_groups == 0 || 32 * o.adj_groups <= B)) {
            s = adjoint_impl<F>(ctx, m, h_src, B, d_T, n_rec, h_rec, d_R, ctx->tune_tau.p, &o,
                                it.data());
            if (s != TT_OK && s != TT_ENOTCONVERGED) return s;
            ms = ctx->stats[TT_STATS_ADJOINT].sweep_ms;
            if (ms < best) {
                best = ms;
                best_c = c;
            }
        }
        if (h_ms) h_ms[c] = ms;
    }
    ctx->tuned_adj.push_back({B, m->dtype, kAdjTuneChunk[best_c], kAdjTuneGroups[best_c]});
    opts->adj_chunk = kAdjTuneChunk[best_c];
    opts->adj_groups = kAdjTuneGroups[best_c];
    return TT_OK;
}

}  // namespace

extern "C" tt_status tt_autotune_adjoint(tt_ctx *ctx, const tt_model *model,
                                         const tt_point *h_src, int n_src, const void *d_T,
                                         int n_rec, const tt_point *h_rec, const double *d_R,
                                         tt_opts *opts, double *h_ms) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if ((s = check_sources(ctx, h_src, n_src)) != TT_OK) return s;
    if ((s = check_opts(ctx, opts)) != TT_OK) return s;
    if (!d_T || !d_R || !h_rec || n_rec < 1)
        return fail(ctx, TT_EINVAL, "tt_autotune_adjoint: NULL argument or no receivers");
    for (const auto &t : ctx->tuned_adj)
        if (t.n_src == n_src && t.dtype == model->dtype) {
            opts->adj_chunk = t.chunk;
            opts->adj_groups = t.groups;
            if (h_ms)
                for (int c = 0; c < kAdjTuneCandidates; ++c) h_ms[c] = 0.0;
            return TT_OK;
        }
    return model->dtype == TT_F32
               ? autotune_adjoint_impl<float>(ctx, model, h_src, n_src, d_T, n_rec, h_rec, d_R,
                                              opts, h_ms)
               : autotune_adjoint_impl<double>(ctx, model, h_src, n_src, d_T, n_rec, h_rec, d_R,
                                               opts, h_ms);
}

// ---------------------------------------------------------------- warm-start network

namespace {

template <typename F>
tt_status net_features_impl(tt_ctx *ctx, const tt_model *m, const tt_point *h_src, int B,
                            float *d_x) {
    tt_status s;
    ENSURE(ctx->pts, sizeof(PointD) * (size_t)B);
    Work<F> W;
    if ((s = work_from_ctx<F>(ctx, W, B, 0)) != TT_OK) return s;
    if ((s = stage_to(ctx, h_src, B, W.src_pts)) != TT_OK) return s;
    if ((s = enq_sources<F>(ctx, W, m, B)) != TT_OK) return s;
    const GeoTab<F> &t = geo<F>(ctx);
    CK(run_net_features<F>(ctx->g, net_grid(ctx), B, 0, B, W.src, W.tabT, W.tabP, t.rad, t.cost,
                           (const F *)m->d_s, (const F *)m->d_xi, (const F *)m->d_eta, d_x,
                           ctx->st));
    ctx->launches += 1;
    CK(cudaStreamSynchronize(ctx->st));
    return TT_OK;
}

// The start of opts.init = 2 without the sweep: the network's tau and the fixed sets.
template <typename F>
tt_status net_start_impl(tt_ctx *ctx, const tt_model *m, const tt_point *h_src, int B,
                         void *d_tau) {
    tt_status s;
    ENSURE(ctx->pts, sizeof(PointD) * (size_t)B);
    Work<F> W;
    if ((s = work_from_ctx<F>(ctx, W, B, 0)) != TT_OK) return s;
    if ((s = net_work_from_ctx<F>(ctx, W, B)) != TT_OK) return s;
    if ((s = stage_to(ctx, h_src, B, W.src_pts)) != TT_OK) return s;
    if ((s = enq_sources<F>(ctx, W, m, B)) != TT_OK) return s;
    CK(cudaMemsetAsync(W.flags + 3, 0, sizeof(int), ctx->st));
    if ((s = enq_warm_start<F>(ctx, W, m, B, (F *)d_tau, kDefaultSpinNs)) != TT_OK) return s;
    CK(run_tau_init<F>(ctx->g, B, W.src, (F *)d_tau, false, ctx->st));
    ctx->launches += 1;
    int h_err = 0;
    CK(cudaMemcpyAsync(&h_err, W.flags + 3, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h_err) return fail(ctx, TT_ETIMEOUT, "tt_net_start: a device-side wait exceeded its limit");
    return TT_OK;
}

}  // namespace

extern "C" {

int tt_net_param_count(void) { return net_param_count(); }

tt_status tt_net_set_stride(tt_ctx *ctx, int stride) {
    if (!ctx) return TT_EINVAL;
    if (stride != 1 && stride != 2)
        return fail(ctx, TT_EINVAL, "tt_net_set_stride: stride %d is not 1 or 2", stride);
    ctx->net_stride = stride;
    return TT_OK;
}

int tt_net_nodes(const tt_ctx *ctx) { return ctx ? (int)net_nodes(ctx) : 0; }

tt_status tt_net_start(tt_ctx *ctx, const tt_model *model, const tt_point *h_src, int n_src,
                       void *d_tau) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if ((s = check_sources(ctx, h_src, n_src)) != TT_OK) return s;
    if (!d_tau) return fail(ctx, TT_EINVAL, "tt_net_start: NULL output");
    if (!ctx->has_net) return fail(ctx, TT_EINVAL, "tt_net_start: no weights (tt_net_set_weights)");
    return model->dtype == TT_F32 ? net_start_impl<float>(ctx, model, h_src, n_src, d_tau)
                                  : net_start_impl<double>(ctx, model, h_src, n_src, d_tau);
}

tt_status tt_net_set_weights(tt_ctx *ctx, const float *d_theta) {
    if (!ctx) return TT_EINVAL;
    if (!d_theta) return fail(ctx, TT_EINVAL, "tt_net_set_weights: NULL weights");
    const int P = net_param_count();
    ENSURE(ctx->net_theta, sizeof(float) * P);
    ENSURE(ctx->net_wbf, sizeof(__nv_bfloat16) * net_weight_image_elems());
    CK(run_round_bf16(P, d_theta, (float *)ctx->net_theta.p, ctx->st));
    CK(run_net_weight_images((const float *)ctx->net_theta.p, (__nv_bfloat16 *)ctx->net_wbf.p,
                             ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->launches += 1 + kNetLayers;
    ctx->has_net = true;
    return TT_OK;
}

tt_status tt_net_infer(tt_ctx *ctx, const float *d_x, int n_grids, float *d_y) {
    if (!ctx) return TT_EINVAL;
    if (!d_x || !d_y || n_grids < 1)
        return fail(ctx, TT_EINVAL, "tt_net_infer: NULL buffer or n_grids < 1");
    if (!ctx->has_net) return fail(ctx, TT_EINVAL, "tt_net_infer: no weights (tt_net_set_weights)");
    const size_t M = net_grid_rows(ctx) * n_grids;
    ENSURE(ctx->net_a, sizeof(__nv_bfloat16) * kNetHidden * M);
    ENSURE(ctx->net_b, sizeof(__nv_bfloat16) * kNetHidden * M);
    ENSURE(ctx->flags, kFlagInts * sizeof(int));
    int *err = (int *)ctx->flags.p + 3;
    CK(cudaMemsetAsync(err, 0, sizeof(int), ctx->st));
    CK(run_net_infer(net_dims(ctx, n_grids), (const float *)ctx->net_theta.p,
                     (const __nv_bfloat16 *)ctx->net_wbf.p, d_x, (__nv_bfloat16 *)ctx->net_a.p,
                     (__nv_bfloat16 *)ctx->net_b.p, d_y, ctx->n_sm, err, kDefaultSpinNs, ctx->st));
    ctx->launches += 1 + kNetLayers;
    int h_err = 0;
    CK(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h_err) return fail(ctx, TT_ETIMEOUT, "tt_net_infer: a device-side wait exceeded its limit");
    return TT_OK;
}

tt_status tt_net_features(tt_ctx *ctx, const tt_model *model, const tt_point *h_src, int n_src,
                          float *d_x) {
    if (!ctx) return TT_EINVAL;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if ((s = check_sources(ctx, h_src, n_src)) != TT_OK) return s;
    if (!d_x) return fail(ctx, TT_EINVAL, "tt_net_features: NULL output");
    return model->dtype == TT_F32 ? net_features_impl<float>(ctx, model, h_src, n_src, d_x)
                                  : net_features_impl<double>(ctx, model, h_src, n_src, d_x);
}

tt_status tt_net_forward(tt_ctx *ctx, const float *d_theta, const float *d_x, int n_grids,
                         float *d_y) {
    if (!ctx) return TT_EINVAL;
    if (!d_theta || !d_x || !d_y || n_grids < 1)
        return fail(ctx, TT_EINVAL, "tt_net_forward: NULL buffer or n_grids < 1");
    const size_t M = (size_t)net_nodes(ctx) * n_grids;
    ENSURE(ctx->net_a, sizeof(float) * kNetHidden * M);
    ENSURE(ctx->net_b, sizeof(float) * kNetHidden * M);
    const ConvDims d = net_dims(ctx, n_grids);
    tt_status s = enq_net_forward(ctx, d_theta, d_x, d, (float *)ctx->net_a.p,
                                  (float *)ctx->net_b.p, (float *)ctx->net_a.p, d_y);
    if (s != TT_OK) return s;
    CK(cudaStreamSynchronize(ctx->st));
    return TT_OK;
}

tt_status tt_net_loss_grad(tt_ctx *ctx, const float *d_theta, const float *d_x,
                           const float *d_target, const float *d_mask, int n_grids,
                           float *d_grad, double *h_loss) {
    if (!ctx) return TT_EINVAL;
    if (!d_theta || !d_x || !d_target || !d_mask || !d_grad || n_grids < 1)
        return fail(ctx, TT_EINVAL, "tt_net_loss_grad: NULL buffer or n_grids < 1");
    const size_t M = (size_t)net_nodes(ctx) * n_grids;
    ENSURE(ctx->net_a, sizeof(float) * kNetHidden * M * 3);
    ENSURE(ctx->net_y, sizeof(float) * M);
    ENSURE(ctx->net_dy, sizeof(float) * M);
    ENSURE(ctx->net_d1, sizeof(float) * kNetHidden * M);
    ENSURE(ctx->net_d2, sizeof(float) * kNetHidden * M);
    ENSURE(ctx->net_wt, sizeof(float) * 27 * kNetHidden * kNetHidden);
    ENSURE(ctx->net_part, sizeof(float) * wgrad_partial_floats());
    ENSURE(ctx->net_scr, sizeof(double) * 4096);
    if (!ctx->h_loss) CK(cudaMallocHost((void **)&ctx->h_loss, sizeof(double)));
    float *a[3] = {(float *)ctx->net_a.p, (float *)ctx->net_a.p + kNetHidden * M,
                   (float *)ctx->net_a.p + 2 * kNetHidden * M};
    float *y = (float *)ctx->net_y.p, *dy = (float *)ctx->net_dy.p;
    float *wt = (float *)ctx->net_wt.p, *part = (float *)ctx->net_part.p;
    double *scr = (double *)ctx->net_scr.p, *loss = scr + 4000;
    const ConvDims d = net_dims(ctx, n_grids);
    tt_status s = enq_net_forward(ctx, d_theta, d_x, d, a[0], a[1], a[2], y);
    if (s != TT_OK) return s;
    CK(run_mse((long long)M, y, d_target, d_mask, dy, scr, loss, ctx->st));
    // backward, last layer first: weight gradient of layer l from its input and the
    // gradient of its output; the gradient of its input through the transposed
    // convolution and the ReLU derivative of the previous layer
    const float *gout = dy;
    float *bufs[2] = {(float *)ctx->net_d1.p, (float *)ctx->net_d2.p};
    for (int l = kNetLayers - 1; l >= 0; --l) {
        const int ci = kNetCin[l], co = kNetCout[l];
        const float *in = l == 0 ? d_x : a[l - 1];
        float *gw = d_grad + net_weight_offset(l);
        CK(run_conv3d_wgrad(d, ci, co, in, l > 0, gout, part, gw, gw + 27 * ci * co, ctx->st));
        if (l > 0) {
            const float *w = d_theta + net_weight_offset(l);
            CK(run_conv3d_flip(ci, co, w, wt, ctx->st));
            float *gin = bufs[l & 1];
            CK(run_conv3d(d, co, ci, gout, false, wt, nullptr, a[l - 1], gin, ctx->st));
            gout = gin;
        }
    }
    ctx->launches += 3 + 2 * kNetLayers + 2 * (kNetLayers - 1);
    CK(cudaMemcpyAsync(ctx->h_loss, loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h_loss) *h_loss = *ctx->h_loss;
    return TT_OK;
}

tt_status tt_net_loss_grad_tc(tt_ctx *ctx, const float *d_theta, const float *d_x,
                              const float *d_target, const float *d_mask, int n_grids,
                              float *d_grad, double *h_loss) {
    if (!ctx) return TT_EINVAL;
    if (!d_theta || !d_x || !d_target || !d_mask || !d_grad || n_grids < 1)
        return fail(ctx, TT_EINVAL, "tt_net_loss_grad_tc: NULL buffer or n_grids < 1");
    const ConvDims d = net_dims(ctx, n_grids);
    const size_t M = (size_t)net_nodes(ctx) * n_grids;
    ENSURE(ctx->net_img, sizeof(__nv_bfloat16) * net_weight_image_elems());
    ENSURE(ctx->net_timg, sizeof(__nv_bfloat16) * net_tweight_image_elems());
    ENSURE(ctx->net_wt, sizeof(float) * 27 * kNetHidden * kNetHidden);
    ENSURE(ctx->net_rows, sizeof(__nv_bfloat16) * net_train_row_elems(d));
    ENSURE(ctx->net_y, sizeof(float) * M);
    ENSURE(ctx->net_dy, sizeof(float) * M);
    ENSURE(ctx->net_part, sizeof(float) * wgrad_partial_floats());
    ENSURE(ctx->net_scr, sizeof(double) * 4096);
    ENSURE(ctx->flags, kFlagInts * sizeof(int));
    if (!ctx->h_loss) CK(cudaMallocHost((void **)&ctx->h_loss, sizeof(double)));
    int *err = (int *)ctx->flags.p + 3;
    double *loss = (double *)ctx->net_scr.p + 4000;
    CK(cudaMemsetAsync(err, 0, sizeof(int), ctx->st));
    CK(run_net_loss_grad_tc(d, d_theta, d_x, d_target, d_mask, d_grad, loss,
                            (__nv_bfloat16 *)ctx->net_img.p, (__nv_bfloat16 *)ctx->net_timg.p,
                            (float *)ctx->net_wt.p, (__nv_bfloat16 *)ctx->net_rows.p,
                            (float *)ctx->net_y.p, (float *)ctx->net_dy.p,
                            (float *)ctx->net_part.p, (double *)ctx->net_scr.p, ctx->n_sm, err,
                            kDefaultSpinNs, ctx->st));
    ctx->launches += 2 + 2 * (kNetLayers - 1) + kNetLayers + 2 + 2 * kNetLayers + (kNetLayers - 1);
    int h_err = 0;
    CK(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(ctx->h_loss, loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h_err)
        return fail(ctx, TT_ETIMEOUT, "tt_net_loss_grad_tc: a device-side wait exceeded its limit");
    if (h_loss) *h_loss = *ctx->h_loss;
    return TT_OK;
}

tt_status tt_net_adam(tt_ctx *ctx, float *d_theta, const float *d_grad, float *d_m, float *d_v,
                      int step, float lr, float beta1, float beta2, float eps) {
    if (!ctx) return TT_EINVAL;
    if (!d_theta || !d_grad || !d_m || !d_v || step < 1)
        return fail(ctx, TT_EINVAL, "tt_net_adam: NULL buffer or step < 1");
    CK(run_adam(net_param_count(), d_theta, d_grad, d_m, d_v, step, lr, beta1, beta2, eps,
                ctx->st));
    ctx->launches += 1;
    CK(cudaStreamSynchronize(ctx->st));
    return TT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- plans (graph-captured steps)

struct tt_plan {
    tt_ctx *ctx = nullptr;
    tt_model model;
    tt_data data;
    tt_opts opts;
    int B = 0, n_rec = 0;
    void *tau = nullptr, *T = nullptr, *P = nullptr;
    double *chi = nullptr, *R = nullptr, *K[3] = {nullptr, nullptr, nullptr};
    // common-receiver terms (Eq. 4, A4) inside the graph: their data, the receiver-time table
    // they read and the sources' shares of chi_cr (has_cr = 0: none)
    int has_cr = 0;
    tt_cr_data cr;
    double *Tr = nullptr, *chi_cr = nullptr;
    int *cr_bad = nullptr;
    std::vector<void *> allocs;
    std::vector<PointD> h_src;
    Work<float> wf;
    Work<double> wd;
    // batch order of the forward (opts.fwd_order = 0): perm[q] = the source at position q; the
    // ordered batch's source points, set-up, iteration counts and tau
    int ordered = 0;
    int *perm = nullptr, *iters_o = nullptr, *conv_o = nullptr;
    PointD *src_pts_o = nullptr;
    SrcC *src_o = nullptr;
    void *tabT_o = nullptr, *tabP_o = nullptr, *tau_o = nullptr;
    // the adjoint's order (its own previous counts): perm_a, the ordered residuals and P; the
    // ordered set-up, counts and T reuse the forward's buffers, free by then
    int *perm_a = nullptr;
    double *R_o = nullptr;
    void *P_o = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches_per_run = 0;  // kernels in the graph, added to ctx->launches per run
};

namespace {

template <typename F> tt_status plan_alloc(tt_plan *p, Work<F> &W) {
    tt_ctx *ctx = p->ctx;
    const GridC &g = ctx->g;
    const int B = p->B, S = 8 * p->n_rec;
    auto get = [&](size_t bytes, void **out) -> tt_status {
        void *q = nullptr;
        if (cudaMalloc(&q, bytes < 256 ? 256 : bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, TT_ENOMEM, "plan workspace allocation of %zu bytes failed", bytes);
        }
        p->allocs.push_back(q);
        *out = q;
        return TT_OK;
    };
    tt_status s;
    W.t0c_slice = factor_slice(g, B, sizeof(F));
    const size_t coef_bytes = sizeof(Vec4<F>) * (size_t)g.N * B;
    W.coef_ok = coef_bytes <= kCoefBudgetBytes;
#define TTGB_GET(field, bytes)                                              \
    do {                                                                    \
        void *q_;                                                           \
        if ((s = get((bytes), &q_)) != TT_OK) return s;                     \
        W.field = reinterpret_cast<decltype(W.field)>(q_);                  \
    } while (0)
    TTGB_GET(src_pts, sizeof(PointD) * B);
    TTGB_GET(rec_pts, sizeof(PointD) * p->n_rec);
    TTGB_GET(src, sizeof(SrcC) * B);
    TTGB_GET(tabT, sizeof(Vec2<F>) * (size_t)g.nt * B);
    TTGB_GET(tabP, sizeof(Vec2<F>) * (size_t)g.np * B);
    TTGB_GET(rec, sizeof(NodeRec<F>) * (size_t)g.N);
    TTGB_GET(t0c, sizeof(Vec4<F>) * (size_t)g.N * W.t0c_slice);
    if (W.coef_ok) TTGB_GET(coef, coef_bytes);
    TTGB_GET(partial, partial_bytes(ctx, B, sizeof(F)));
    TTGB_GET(conv_f, sizeof(int) * B);
    TTGB_GET(iters_f, sizeof(int) * B);
    TTGB_GET(conv_a, sizeof(int) * B);
    TTGB_GET(iters_a, sizeof(int) * B);
    TTGB_GET(nact, sizeof(int) * kMaxBarrierGroups);
    TTGB_GET(flags, kFlagInts * sizeof(int));
    TTGB_GET(bar, sizeof(BarrierState) * kMaxBarrierGroups);
    TTGB_GET(cq, sizeof(long long) * S);
    TTGB_GET(wq, sizeof(double) * S);
    TTGB_GET(sidx, sizeof(int) * (size_t)g.N);
    TTGB_GET(next, sizeof(int) * S);
    TTGB_GET(heads, sizeof(int) * S);
    TTGB_GET(nheads, sizeof(int));
    TTGB_GET(JS, sizeof(F) * (size_t)S * B);
    if (p->has_cr) {
        void *q_;
        if ((s = get(sizeof(int), &q_)) != TT_OK) return s;
        p->cr_bad = (int *)q_;
    }
    const int n_slots = refill_slots_for(&p->opts, B, W.t0c_slice);
    if (n_slots > 0) {
        TTGB_GET(tau_w, sizeof(F) * (size_t)g.N * n_slots);
        TTGB_GET(slot_srcc, sizeof(SrcC) * (size_t)n_slots);
        TTGB_GET(slot_int, sizeof(int) * (4 * (size_t)n_slots + 1));
        W.n_slots = n_slots;
    }
    if (p->ordered) {
        void *q_;
#define TTGB_PGET(field, type, bytes)                                        \
    do {                                                                     \
        if ((s = get((bytes), &q_)) != TT_OK) return s;                      \
        p->field = reinterpret_cast<type>(q_);                               \
    } while (0)
        TTGB_PGET(perm, int *, sizeof(int) * B);
        TTGB_PGET(iters_o, int *, sizeof(int) * B);
        TTGB_PGET(conv_o, int *, sizeof(int) * B);
        TTGB_PGET(src_pts_o, PointD *, sizeof(PointD) * B);
        TTGB_PGET(src_o, SrcC *, sizeof(SrcC) * B);
        TTGB_PGET(tabT_o, void *, sizeof(Vec2<F>) * (size_t)g.nt * B);
        TTGB_PGET(tabP_o, void *, sizeof(Vec2<F>) * (size_t)g.np * B);
        TTGB_PGET(tau_o, void *, sizeof(F) * (size_t)g.N * B);
        TTGB_PGET(perm_a, int *, sizeof(int) * B);
        TTGB_PGET(R_o, double *, sizeof(double) * (size_t)B * (p->n_rec > 0 ? p->n_rec : 1));
        TTGB_PGET(P_o, void *, sizeof(F) * (size_t)g.N * B);
#undef TTGB_PGET
    }
    if (p->opts.init == 2) {
        W.net_chunk = net_chunk(ctx, B);
        const size_t Nn = (size_t)net_nodes(ctx);
        TTGB_GET(net_x, sizeof(float) * kNetFeatures * Nn * W.net_chunk);
        TTGB_GET(net_a, sizeof(__nv_bfloat16) * kNetHidden * net_grid_rows(ctx) * W.net_chunk);
        TTGB_GET(net_b, sizeof(__nv_bfloat16) * kNetHidden * net_grid_rows(ctx) * W.net_chunk);
        TTGB_GET(net_y, sizeof(float) * Nn * W.net_chunk);
        W.net_theta = (const float *)ctx->net_theta.p;
        W.net_wbf = (const __nv_bfloat16 *)ctx->net_wbf.p;
    }
#undef TTGB_GET
    return TT_OK;
}

// Everything one step enqueues, in order; captured once into the plan's graph.
template <typename F> tt_status plan_enqueue(tt_plan *p, Work<F> &W) {
    tt_ctx *ctx = p->ctx;
    const GridC &g = ctx->g;
    tt_status s;
    CK(cudaMemsetAsync(W.flags, 0, 4 * sizeof(int), ctx->st));
    if ((s = enq_receivers(ctx, W.rec_pts, p->n_rec, W.cq, W.wq, W.flags)) != TT_OK) return s;
    if ((s = enq_sources<F>(ctx, W, &p->model, p->B)) != TT_OK) return s;
    if (p->ordered) {
        Work<F> Wo = W;
        Wo.src_pts = p->src_pts_o;
        Wo.src = p->src_o;
        Wo.tabT = (Vec2<F> *)p->tabT_o;
        Wo.tabP = (Vec2<F> *)p->tabP_o;
        Wo.iters_f = p->iters_o;
        Wo.conv_f = p->conv_o;
        if ((s = enq_forward_ordered<F>(ctx, W, Wo, p->perm, &p->model, p->B, p->tau, p->tau_o,
                                        p->T, &p->opts)) != TT_OK)
            return s;
    } else if ((s = enq_forward<F>(ctx, W, &p->model, p->B, p->tau, p->T, &p->opts)) != TT_OK) {
        return s;
    }
    if ((s = enq_readback(ctx, p->B, W.iters_f, W.conv_f, W.flags, W.bar, TT_STATS_FORWARD)) !=
        TT_OK)
        return s;
    if ((s = enq_misfit(ctx, p->T, p->model.dtype, &p->data, W.cq, W.wq, W.flags, p->Tr, p->chi,
                        p->R)) != TT_OK)
        return s;
    if (p->has_cr) {  // Eq. 4 terms and their adjoint source (A4), added into R
        CK(run_misfit_cr(p->cr.n_src, p->cr.n_rec, p->cr.d_off, p->cr.d_other, p->cr.d_dtobs,
                         p->cr.d_w, p->cr.gamma, p->Tr, p->chi_cr, p->R, p->cr_bad, ctx->st));
        ctx->launches += 1;
    }
    if (p->ordered) {
        // the adjoint over the batch ordered by the previous run's adjoint counts: T, R and
        // the set-up in that order, then P and the counts back in the batch's order
        Work<F> Wa = W;
        Wa.src_pts = p->src_pts_o;
        Wa.src = p->src_o;
        Wa.tabT = (Vec2<F> *)p->tabT_o;
        Wa.tabP = (Vec2<F> *)p->tabP_o;
        Wa.iters_a = p->iters_o;
        Wa.conv_a = p->conv_o;
        CK(run_gather_points(p->B, p->perm_a, W.src_pts, Wa.src_pts, ctx->st));
        if ((s = enq_sources<F>(ctx, Wa, &p->model, p->B)) != TT_OK) return s;
        CK(run_permute_rows<F>(g.N, p->B, p->perm_a, (F *)p->T, (F *)p->tau_o, true, ctx->st));
        CK(run_gather_rows(p->B, p->n_rec, p->perm_a, p->R, p->R_o, ctx->st));
        if ((s = enq_adjoint<F>(ctx, Wa, &p->model, p->B, p->tau_o, p->n_rec, p->R_o, p->P_o,
                                &p->opts)) != TT_OK)
            return s;
        CK(run_permute_rows<F>(g.N, p->B, p->perm_a, (F *)p->P, (F *)p->P_o, false, ctx->st));
        CK(run_unpermute_ints(p->B, p->perm_a, p->iters_o, p->conv_o, W.iters_a, W.conv_a,
                              ctx->st));
        ctx->launches += 5;
    } else if ((s = enq_adjoint<F>(ctx, W, &p->model, p->B, p->T, p->n_rec, p->R, p->P,
                                   &p->opts)) != TT_OK) {
        return s;
    }
    for (int q = 0; q < 3; ++q)
        CK(cudaMemsetAsync(p->K[q], 0, sizeof(double) * (size_t)g.N, ctx->st));
    if ((s = enq_kernel(ctx, &p->model, p->B, p->T, p->P, p->K[0], p->K[1], p->K[2])) != TT_OK)
        return s;
    if (p->ordered) {  // the next run's orders: this run's counts, fewest first
        CK(run_order_update(p->B, W.iters_f, p->perm, ctx->st));
        CK(run_order_update(p->B, W.iters_a, p->perm_a, ctx->st));
        ctx->launches += 2;
    }
    return enq_readback(ctx, p->B, W.iters_a, W.conv_a, W.flags, W.bar, TT_STATS_ADJOINT);
}

template <typename F> tt_status plan_build(tt_plan *p, Work<F> &W, const tt_point *h_src) {
    tt_ctx *ctx = p->ctx;
    tt_status s;
    if ((s = plan_alloc<F>(p, W)) != TT_OK) return s;
    if (p->ordered) {
        CK(run_order_identity(p->B, p->perm, ctx->st));
        CK(run_order_identity(p->B, p->perm_a, ctx->st));
    }
    if ((s = stage_to(ctx, p->data.h_rec, p->n_rec, W.rec_pts)) != TT_OK) return s;
    if ((s = stage_to(ctx, h_src, p->B, W.src_pts)) != TT_OK) return s;
    CK(cudaStreamSynchronize(ctx->st));
    // Sizes and launch shapes are decided on the host while capturing; the kernels and copies
    // go into the graph. The legacy default stream cannot be captured, so the capture runs on
    // a private stream; the graph is launched on the context's stream.
    cudaStream_t cap = nullptr;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t own = ctx->st;
    ctx->st = cap;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    cudaGraph_t graph = nullptr;
    const long long launches0 = ctx->launches;
    if (e == cudaSuccess) {
        s = plan_enqueue<F>(p, W);
        e = cudaStreamEndCapture(cap, &graph);
    }
    p->launches_per_run = ctx->launches - launches0;
    ctx->launches = launches0;
    ctx->st = own;
    cudaStreamDestroy(cap);
    if (s != TT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess)
        return fail(ctx, TT_ECUDA, "stream capture of the step failed: %s", cudaGetErrorString(e));
    p->graph = graph;
    CK(cudaGraphInstantiate(&p->exec, graph, 0));
    return TT_OK;
}

}  // namespace

extern "C" {

tt_status tt_plan_create_cr(tt_plan **out, tt_ctx *ctx, const tt_model *model,
                            const tt_point *h_src, int n_src, const tt_data *data,
                            const tt_cr_data *cr, const tt_opts *opts, void *d_tau, void *d_T,
                            void *d_P, double *d_chi, double *d_Tr, double *d_chi_cr,
                            double *d_R, double *d_Ks, double *d_Kxi, double *d_Keta);

tt_status tt_plan_create(tt_plan **out, tt_ctx *ctx, const tt_model *model,
                         const tt_point *h_src, int n_src, const tt_data *data,
                         const tt_opts *opts, void *d_tau, void *d_T, void *d_P, double *d_chi,
                         double *d_R, double *d_Ks, double *d_Kxi, double *d_Keta) {
    return tt_plan_create_cr(out, ctx, model, h_src, n_src, data, nullptr, opts, d_tau, d_T,
                             d_P, d_chi, nullptr, nullptr, d_R, d_Ks, d_Kxi, d_Keta);
}

tt_status tt_plan_create_cr(tt_plan **out, tt_ctx *ctx, const tt_model *model,
                            const tt_point *h_src, int n_src, const tt_data *data,
                            const tt_cr_data *cr, const tt_opts *opts, void *d_tau, void *d_T,
                            void *d_P, double *d_chi, double *d_Tr, double *d_chi_cr,
                            double *d_R, double *d_Ks, double *d_Kxi, double *d_Keta) {
    if (!out || !ctx) return TT_EINVAL;
    *out = nullptr;
    tt_status s;
    if ((s = check_model(ctx, model)) != TT_OK) return s;
    if ((s = check_sources(ctx, h_src, n_src)) != TT_OK) return s;
    if ((s = check_opts(ctx, opts)) != TT_OK) return s;
    if ((s = check_data(ctx, data)) != TT_OK) return s;
    if (data->n_src != n_src) return fail(ctx, TT_EINVAL, "data describe %d sources, not %d",
                                          data->n_src, n_src);
    if (!d_tau || !d_T || !d_P || !d_R || !d_Ks || !d_Kxi || !d_Keta)
        return fail(ctx, TT_EINVAL, "tt_plan_create: NULL buffer");
    if (cr) {
        if (!d_Tr || !d_chi_cr || !cr->d_off)
            return fail(ctx, TT_EINVAL, "tt_plan_create_cr: NULL argument");
        if (cr->n_src != n_src || cr->n_rec != data->n_rec)
            return fail(ctx, TT_EINVAL, "tt_plan_create_cr: cr data for %d sources and %d "
                        "receivers, the batch has %d and %d", cr->n_src, cr->n_rec, n_src,
                        data->n_rec);
        if (cr->n_entries > 0) {
            if (!cr->d_other || !cr->d_dtobs || !cr->d_w)
                return fail(ctx, TT_EINVAL, "tt_plan_create_cr: NULL entry arrays");
            // every entry must name a source of the batch: checked once, on the host
            std::vector<int> other(cr->n_entries);
            CK(cudaMemcpy(other.data(), cr->d_other, sizeof(int) * other.size(),
                          cudaMemcpyDeviceToHost));
            for (int q : other)
                if (q < 0 || q >= n_src)
                    return fail(ctx, TT_EINVAL, "tt_plan_create_cr: an entry names source %d "
                                "outside the batch", q);
        }
    }
    tt_plan *p = new tt_plan();
    if (cr) {
        p->has_cr = 1;
        p->cr = *cr;
        p->Tr = d_Tr;
        p->chi_cr = d_chi_cr;
    }
    p->ctx = ctx;
    p->model = *model;
    p->data = *data;
    p->opts = *opts;
    p->B = n_src;
    p->n_rec = data->n_rec;
    p->tau = d_tau;
    p->T = d_T;
    p->P = d_P;
    p->chi = d_chi;
    p->R = d_R;
    p->K[0] = d_Ks;
    p->K[1] = d_Kxi;
    p->K[2] = d_Keta;
    p->h_src.resize(n_src);
    for (int b = 0; b < n_src; ++b)
        p->h_src[b] = PointD{h_src[b].depth_km, h_src[b].lat_deg, h_src[b].lon_deg};
    // the batch order matters where the sweep runs several barrier groups side by side
    p->ordered = opts->fwd_order == 0 && opts->fwd_slots == 0 && n_src >= 64;
    s = model->dtype == TT_F32 ? plan_build<float>(p, p->wf, h_src)
                               : plan_build<double>(p, p->wd, h_src);
    if (s != TT_OK) {
        tt_plan_destroy(p);
        return s;
    }
    *out = p;
    return TT_OK;
}

tt_status tt_plan_run(tt_plan *p, int *h_iters_fwd, int *h_iters_adj) {
    if (!p) return TT_EINVAL;
    tt_ctx *ctx = p->ctx;
    CK(cudaGraphLaunch(p->exec, ctx->st));
    ctx->launches += p->launches_per_run;
    CK(cudaStreamSynchronize(ctx->st));
    Readback r = readback_view(ctx);
    if (r.flags[1]) return fail(ctx, TT_EINVAL, "tt_plan_run: receiver index out of range");
    if (r.flags[2]) return fail(ctx, TT_EINVAL, "tt_plan_run: receiver outside the grid");
    ctx->warm_last = p->opts.init == 2;
    ctx->scheme_last = p->opts.scheme;
    tt_status sf = solve_status(ctx, p->B, p->h_src.data(), h_iters_fwd, p->opts.max_iter_fwd,
                                "tt_plan_run (forward)", TT_STATS_FORWARD);
    if (sf != TT_OK && sf != TT_ENOTCONVERGED) return sf;
    tt_status sa = solve_status(ctx, p->B, p->h_src.data(), h_iters_adj, p->opts.max_iter_adj,
                                "tt_plan_run (adjoint)", TT_STATS_ADJOINT);
    return sa != TT_OK ? sa : sf;
}

void tt_plan_destroy(tt_plan *p) {
    if (!p) return;
    if (p->ctx && p->ctx->st) cudaStreamSynchronize(p->ctx->st);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (void *q : p->allocs) cudaFree(q);
    delete p;
}

}  // extern "C"
