// C ABI of libttgb (declared in include/tt.h): context, validation, workspace and the
// orchestration of the kernels in tt_sweep.cu and tt_aux.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <vector>

#include "tt.h"
#include "tt_aux.h"
#include "tt_internal.h"

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
    DevBuf src, pts, tabT, tabP, rec, partial, conv, iters, nact, bar, flags;
    DevBuf cq, wq, sidx, next, heads, nheads, JS, coef, t0c;
    int *h_pinned = nullptr;  // readback: [0..TT_MAX_BATCH) iterations, then flags
    PointD *h_pts = nullptr;  // staging for source / receiver positions
    size_t h_pts_cap = 0;

    cudaEvent_t ev_start[2] = {nullptr, nullptr}, ev_stop[2] = {nullptr, nullptr};
    tt_stats stats[2] = {};
    long long launches = 0;   // kernels launched by this context
};

namespace {

constexpr long long kDefaultSpinNs = 2000000000LL;
// Largest per-(node, source) coefficient array the adjoint keeps in its workspace.
constexpr size_t kCoefBudgetBytes = 64ull << 30;
// Largest factor cache (1/T0 and grad T0 / T0 per node and source) one forward slice keeps.
constexpr size_t kFactorCacheBudgetBytes = 32ull << 30;

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

tt_status stage_points(tt_ctx *ctx, const tt_point *h, int n, DevBuf &dst) {
    if ((size_t)n > ctx->h_pts_cap) {
        if (ctx->h_pts) cudaFreeHost(ctx->h_pts);
        ctx->h_pts = nullptr;
        ctx->h_pts_cap = 0;
        CK(cudaMallocHost((void **)&ctx->h_pts, sizeof(PointD) * (size_t)n));
        ctx->h_pts_cap = n;
    }
    // The stream may still read the staging buffer from an earlier call.
    CK(cudaStreamSynchronize(ctx->st));
    for (int q = 0; q < n; ++q) ctx->h_pts[q] = PointD{h[q].depth_km, h[q].lat_deg, h[q].lon_deg};
    ENSURE(dst, sizeof(PointD) * (size_t)n);
    CK(cudaMemcpyAsync(dst.p, ctx->h_pts, sizeof(PointD) * (size_t)n, cudaMemcpyHostToDevice,
                       ctx->st));
    return TT_OK;
}

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
    int per_sm = fwd ? forward_blocks_per_sm<F>(block, smem) : adjoint_blocks_per_sm<F>(block, smem);
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
    return TT_OK;
}

unsigned long long spin_ns(const tt_opts *o) {
    return (unsigned long long)(o->spin_limit_ns > 0 ? o->spin_limit_ns : kDefaultSpinNs);
}

// Resets convergence state and the barrier, then launches.
tt_status reset_solver_state(tt_ctx *ctx, int B) {
    ENSURE(ctx->conv, sizeof(int) * (size_t)B);
    ENSURE(ctx->iters, sizeof(int) * (size_t)B);
    ENSURE(ctx->nact, sizeof(int) * kMaxBarrierGroups);
    ENSURE(ctx->bar, sizeof(BarrierState) * kMaxBarrierGroups);
    ENSURE(ctx->flags, 4 * sizeof(int));
    CK(cudaMemsetAsync(ctx->conv.p, 0, sizeof(int) * (size_t)B, ctx->st));
    CK(cudaMemsetAsync(ctx->iters.p, 0, sizeof(int) * (size_t)B, ctx->st));
    CK(cudaMemsetAsync(ctx->nact.p, 0, sizeof(int) * kMaxBarrierGroups, ctx->st));
    CK(cudaMemsetAsync(ctx->bar.p, 0, sizeof(BarrierState) * kMaxBarrierGroups, ctx->st));
    CK(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), ctx->st));
    return TT_OK;
}

// Reads back iterations, convergence flags, the barrier status and the validation flag,
// waits for the stream and turns them into a status.
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

tt_status finish_solve(tt_ctx *ctx, int B, int *h_iters, int max_iter, const char *what,
                       int which) {
    int *h = ctx->h_pinned;
    CK(cudaMemcpyAsync(h, ctx->iters.p, sizeof(int) * (size_t)B, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(h + TT_MAX_BATCH, ctx->conv.p, sizeof(int) * (size_t)B,
                       cudaMemcpyDeviceToHost, ctx->st));
    unsigned char *hb = (unsigned char *)(ctx->h_pinned + 2 * TT_MAX_BATCH + 8);
    CK(cudaMemcpyAsync(hb, ctx->bar.p, sizeof(BarrierState) * kMaxBarrierGroups,
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(h + 2 * TT_MAX_BATCH + 1, ctx->flags.p, sizeof(int),
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h[2 * TT_MAX_BATCH + 1])
        return fail(ctx, TT_EINVAL, "%s: model has s <= 0 or xi^2 + eta^2 >= 1/4", what);
    for (int q = 0; q < kMaxBarrierGroups; ++q) {
        int st;
        memcpy(&st, hb + q * sizeof(BarrierState) + offsetof(BarrierState, status), sizeof st);
        if (st == kDevTimeout)
            return fail(ctx, TT_ETIMEOUT, "%s: a device-side wait exceeded its limit", what);
    }
    if (h_iters) memcpy(h_iters, h, sizeof(int) * (size_t)B);
    {
        tt_stats &S = ctx->stats[which];
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev_start[which], ctx->ev_stop[which]));
        S.sweep_ms = ms;
        const int lo = which == TT_STATS_FORWARD ? 1 : 0;
        long long upd = 0;
        int imax = 0;
        for (int b = 0; b < B; ++b) {
            upd += 8LL * h[b] * updated_nodes(ctx, ctx->h_pts[b], lo);
            imax = h[b] > imax ? h[b] : imax;
        }
        const GridC &g = ctx->g;
        S.node_updates = upd;
        S.iters_max = imax;
        S.node_sweeps = 8LL * imax * (long long)(g.nr - 2 * lo) * (g.nt - 2 * lo) * (g.np - 2 * lo);
    }
    int nc = 0;
    for (int b = 0; b < B; ++b) nc += h[TT_MAX_BATCH + b] == 0;
    if (nc)
        return fail(ctx, TT_ENOTCONVERGED, "%s: %d of %d sources did not converge in %d iterations",
                    what, nc, B, max_iter);
    return TT_OK;
}

template <typename F> GeoTab<F> &geo(tt_ctx *ctx);
template <> GeoTab<float> &geo<float>(tt_ctx *ctx) { return ctx->gf; }
template <> GeoTab<double> &geo<double>(tt_ctx *ctx) { return ctx->gd; }

template <typename F>
tt_status forward_impl(tt_ctx *ctx, const tt_model *m, const tt_point *h_src, int B, void *d_tau,
                       void *d_T, const tt_opts *o, int *h_iters) {
    const GridC &g = ctx->g;
    tt_status s;
    if ((s = stage_points(ctx, h_src, B, ctx->pts)) != TT_OK) return s;
    ENSURE(ctx->src, sizeof(SrcC) * (size_t)B);
    ENSURE(ctx->tabT, sizeof(Vec2<F>) * (size_t)g.nt * B);
    ENSURE(ctx->tabP, sizeof(Vec2<F>) * (size_t)g.np * B);
    ENSURE(ctx->rec, sizeof(NodeRec<F>) * (size_t)g.N);
    if ((s = reset_solver_state(ctx, B)) != TT_OK) return s;
    SrcC *src = (SrcC *)ctx->src.p;
    CK(run_source_setup<F>(g, m->d_s, m->d_xi, m->d_eta, (const PointD *)ctx->pts.p, B, src,
                           (Vec2<F> *)ctx->tabT.p, (Vec2<F> *)ctx->tabP.p, ctx->st));
    CK(run_node_records<F>(g, m->d_s, m->d_xi, m->d_eta, ctx->gd.h2, ctx->gd.cost,
                           (NodeRec<F> *)ctx->rec.p, (int *)ctx->flags.p, ctx->st));
    CK(run_tau_init<F>(g, B, src, (F *)d_tau, o->init == 0, ctx->st));
    ctx->launches += 4 + (o->init == 0 ? 2 : 1);

    // Tile schedules stage 32 sources per task with TMA: they need B >= 32 and rows of tau
    // (B values) that are a multiple of 16 bytes. Automatic: node hyperplanes.
    const bool tiles_ok = B >= 32 && (B * sizeof(F)) % 16 == 0;
    int sched = o->sweep_schedule == 0 ? 1 : o->sweep_schedule;
    if (sched >= 2 && !tiles_ok) sched = 1;
    // Source slices: the factor cache of one slice must fit the workspace budget.
    const size_t per_src = sizeof(Vec4<F>) * (size_t)g.N;
    int slice = B;
    if (per_src * (size_t)B > kFactorCacheBudgetBytes) {
        slice = (int)(kFactorCacheBudgetBytes / per_src) / 32 * 32;
        if (slice < 32) slice = 32;
    }
    ENSURE(ctx->t0c, per_src * (size_t)(slice < B ? slice : B));

    const GeoTab<F> &t = geo<F>(ctx);
    FwdArgs<F> a;
    memset(&a, 0, sizeof a);
    a.g = g;
    a.B = B;
    a.n_planes = ctx->interior.n_planes;
    a.er = (F)(0.5 / g.dr);
    a.rec = (const NodeRec<F> *)ctx->rec.p;
    a.tau = (F *)d_tau;
    a.src = src;
    a.tabT = (const Vec2<F> *)ctx->tabT.p;
    a.tabP = (const Vec2<F> *)ctx->tabP.p;
    a.rad = t.rad;
    a.cost = t.cost;
    a.sint = t.sint;
    a.nodes = ctx->interior.nodes;
    a.off = ctx->interior.off;
    a.bar = (BarrierState *)ctx->bar.p;
    a.conv = (int *)ctx->conv.p;
    a.iters = (int *)ctx->iters.p;
    a.n_active = (int *)ctx->nact.p;
    a.tol = (F)o->tol_fwd;
    a.max_iter = o->max_iter_fwd;
    a.spin_ns = spin_ns(o);
    a.t0c = (Vec4<F> *)ctx->t0c.p;
    a.na = g.nr - 2;
    a.nb = g.nt - 2;
    a.nc = g.np - 2;
    CUtensorMap map_tau, map_rec;
    if (sched >= 2) {
        const TileShape sh = kTileShapes[sched - 2];
        const unsigned box_tau[4] = {32u, (unsigned)sh.tc + 2, (unsigned)sh.tb + 2,
                                     (unsigned)sh.ta + 2};
        const unsigned box_rec[4] = {8u, (unsigned)sh.tc, (unsigned)sh.tb, (unsigned)sh.ta};
        if ((s = encode_map4<F>(ctx, &map_tau, d_tau, B, box_tau)) != TT_OK) return s;
        if ((s = encode_map4<F>(ctx, &map_rec, ctx->rec.p, 8, box_rec)) != TT_OK) return s;
        const TileSchedule &ts = ctx->tiled[sched - 2];
        a.tiles = ts.tiles;
        a.toff = ts.off;
        a.n_tplanes = ts.n_planes;
    }

    int max_grid_used = 0;
    CK(cudaEventRecord(ctx->ev_start[TT_STATS_FORWARD], ctx->st));
    for (int s0 = 0; s0 < B; s0 += slice) {
        const int n = slice < B - s0 ? slice : B - s0;
        a.src_lo = s0;
        a.src_n = n;
        int grid = 0;
        if (sched == 1 || n < 32) {  // a tile task stages 32 sources: short slices use nodes
            // 256-thread blocks; one barrier group per resident block slot of an SM, so
            // each SM interleaves the groups; each group gets a multiple of 32 sources.
            const int block = 256;
            int per_sm = forward_blocks_per_sm<F>(block, (size_t)n * sizeof(F));
            if (per_sm <= 0) return fail(ctx, TT_ECUDA, "sweep kernel cannot be resident");
            if (per_sm > kMaxBarrierGroups) per_sm = kMaxBarrierGroups;
            int max_grid = per_sm * ctx->n_sm;
            if (o->launch_blocks > 0 && o->launch_blocks < max_grid) max_grid = o->launch_blocks;
            int groups = per_sm;
            if (groups > (n + 31) / 32) groups = (n + 31) / 32;
            if (groups > max_grid) groups = max_grid;
            int gsrc = ((n + groups - 1) / groups + 31) / 32 * 32;
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
            ENSURE(ctx->partial, sizeof(F) * 2 * (size_t)B * grid);
            a.partial = (F *)ctx->partial.p;
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
            ENSURE(ctx->partial, sizeof(F) * 2 * (size_t)B * grid);
            a.partial = (F *)ctx->partial.p;
            CUtensorMap map_t0c;
            const TileShape sh = kTileShapes[sched - 2];
            const unsigned box_c[4] = {128u, (unsigned)sh.tc, (unsigned)sh.tb, (unsigned)sh.ta};
            if ((s = encode_map4<F>(ctx, &map_t0c, ctx->t0c.p, 4LL * n, box_c)) != TT_OK) return s;
            CK(launch_t0_cache<F>(a, ctx->st));
            CK(launch_forward_tiled<F>(map_tau, map_rec, map_t0c, a, sched - 2, grid, ctx->st));
            ctx->stats[TT_STATS_FORWARD].block_threads = kTileThreads;
        }
        ctx->launches += 2;
        if (grid > max_grid_used) max_grid_used = grid;
    }
    CK(cudaEventRecord(ctx->ev_stop[TT_STATS_FORWARD], ctx->st));
    ctx->stats[TT_STATS_FORWARD].grid_blocks = max_grid_used;
    if (d_T) {
        CK(run_traveltime<F>(g, B, src, a.tabT, a.tabP, t.rad, t.cost, t.sint, (const F *)d_tau,
                             (F *)d_T, ctx->st));
        ctx->launches += 1;
    }
    return finish_solve(ctx, B, h_iters, o->max_iter_fwd, "tt_forward", TT_STATS_FORWARD);
}

tt_status receivers_impl(tt_ctx *ctx, const tt_point *h_rec, int n_rec) {
    if (n_rec < 1 || !h_rec) return fail(ctx, TT_EINVAL, "need at least one receiver");
    for (int m = 0; m < n_rec; ++m)
        if (!inside(ctx, h_rec[m]))
            return fail(ctx, TT_EINVAL, "receiver %d (%g km, %g, %g) outside the grid", m,
                        h_rec[m].depth_km, h_rec[m].lat_deg, h_rec[m].lon_deg);
    tt_status s;
    if ((s = stage_points(ctx, h_rec, n_rec, ctx->pts)) != TT_OK) return s;
    ENSURE(ctx->cq, sizeof(long long) * 8 * (size_t)n_rec);
    ENSURE(ctx->wq, sizeof(double) * 8 * (size_t)n_rec);
    ENSURE(ctx->flags, 4 * sizeof(int));
    CK(run_receiver_setup(ctx->g, (const PointD *)ctx->pts.p, n_rec, (long long *)ctx->cq.p,
                          (double *)ctx->wq.p, (int *)ctx->flags.p + 2, ctx->st));
    ctx->launches += 1;
    return TT_OK;
}

template <typename F>
tt_status adjoint_impl(tt_ctx *ctx, const tt_model *m, const tt_point *h_src, int B,
                       const void *d_T, int n_rec, const tt_point *h_rec, const double *d_R,
                       void *d_P, const tt_opts *o, int *h_iters) {
    const GridC &g = ctx->g;
    tt_status s;
    if ((s = reset_solver_state(ctx, B)) != TT_OK) return s;
    if ((s = receivers_impl(ctx, h_rec, n_rec)) != TT_OK) return s;
    const int S = 8 * n_rec;
    ENSURE(ctx->sidx, sizeof(int) * (size_t)g.N);
    ENSURE(ctx->next, sizeof(int) * (size_t)S);
    ENSURE(ctx->heads, sizeof(int) * (size_t)S);
    ENSURE(ctx->nheads, sizeof(int));
    ENSURE(ctx->JS, sizeof(F) * (size_t)S * B);
    CK(run_point_sources<F>(g, n_rec, (const long long *)ctx->cq.p, (const double *)ctx->wq.p,
                            (int *)ctx->sidx.p, (int *)ctx->next.p, (int *)ctx->heads.p,
                            (int *)ctx->nheads.p, d_R, B, (F *)ctx->JS.p, ctx->st));
    ctx->launches += 5;
    if ((s = stage_points(ctx, h_src, B, ctx->pts)) != TT_OK) return s;
    ENSURE(ctx->src, sizeof(SrcC) * (size_t)B);
    ENSURE(ctx->tabT, sizeof(Vec2<F>) * (size_t)g.nt * B);
    ENSURE(ctx->tabP, sizeof(Vec2<F>) * (size_t)g.np * B);
    SrcC *src = (SrcC *)ctx->src.p;
    CK(run_source_setup<F>(g, m->d_s, m->d_xi, m->d_eta, (const PointD *)ctx->pts.p, B, src,
                           (Vec2<F> *)ctx->tabT.p, (Vec2<F> *)ctx->tabP.p, ctx->st));
    ctx->launches += 3;
    CK(cudaMemsetAsync(d_P, 0, sizeof(F) * (size_t)g.N * B, ctx->st));

    // Face-coefficient sweep when the per-(node, source) coefficients fit the workspace
    // budget; otherwise the sweep that evaluates the flux velocities at every update.
    const size_t coef_bytes = sizeof(Vec4<F>) * (size_t)g.N * B;
    const bool faces = coef_bytes <= kCoefBudgetBytes;
    int grid, block, slots;
    int n_bgroups = 1, grp_blocks = 0, grp_src = B;
    if (faces) {
        // Source slices of adj_chunk sources, one cooperative launch each, run one after
        // another: a hyperplane of one slice (coefficients of two planes, P of three) then
        // stays in L2. Automatic: slices of at most 128 sources.
        block = 256;
        int chunk = o->adj_chunk > 0 ? o->adj_chunk : 128;
        grp_src = chunk >= B ? B : (chunk + 31) / 32 * 32;
        n_bgroups = (B + grp_src - 1) / grp_src;
        size_t smem = (size_t)grp_src * 2 * sizeof(F);
        int per_sm = adjoint_faces_blocks_per_sm<F>(block, smem);
        if (per_sm <= 0) return fail(ctx, TT_ECUDA, "adjoint sweep cannot be resident");
        if (per_sm > 4) per_sm = 4;
        int max_grid = per_sm * ctx->n_sm;
        if (o->launch_blocks > 0 && o->launch_blocks < max_grid) max_grid = o->launch_blocks;
        grp_blocks = max_grid;
        if ((long long)grp_blocks * block < grp_src) {
            int need = (grp_src + block - 1) / block;
            if (need > per_sm * ctx->n_sm)
                return fail(ctx, TT_EINVAL, "batch of %d sources exceeds one resident launch", B);
            grp_blocks = need;
        }
        grid = grp_blocks;
        slots = 0;
        ENSURE(ctx->coef, coef_bytes);
    } else if ((s = sweep_shape<F>(ctx, false, B, ctx->full, o->launch_blocks, grid, block,
                                   slots)) != TT_OK) {
        return s;
    }
    ENSURE(ctx->partial, sizeof(F) * 2 * (size_t)B * grid);
    const GeoTab<F> &t = geo<F>(ctx);
    AdjArgs<F> a;
    a.g = g;
    a.B = B;
    a.slots = slots;
    a.n_planes = ctx->full.n_planes;
    a.n_rec = n_rec;
    a.T = (const F *)d_T;
    a.P = (F *)d_P;
    a.xi = (const F *)m->d_xi;
    a.eta = (const F *)m->d_eta;
    a.src = src;
    a.cost = t.cost;
    a.costf = t.costf;
    a.h2 = t.h2;
    a.arf = t.arf;
    a.sidx = (const int *)ctx->sidx.p;
    a.JS = (const F *)ctx->JS.p;
    a.nodes = ctx->full.nodes;
    a.off = ctx->full.off;
    a.bar = (BarrierState *)ctx->bar.p;
    a.partial = (F *)ctx->partial.p;
    a.conv = (int *)ctx->conv.p;
    a.iters = (int *)ctx->iters.p;
    a.n_active = (int *)ctx->nact.p;
    a.tol = (F)o->tol_adj;
    a.max_iter = o->max_iter_adj;
    a.spin_ns = spin_ns(o);
    a.coef = faces ? (Vec4<F> *)ctx->coef.p : nullptr;
    a.n_bgroups = n_bgroups;
    a.grp_blocks = grp_blocks;
    a.grp_src = grp_src;
    if (faces) {
        CK(launch_adjoint_coefs<F>(a, ctx->st));
        ctx->launches += 1;
    }
    CK(cudaEventRecord(ctx->ev_start[TT_STATS_ADJOINT], ctx->st));
    if (faces) {
        for (int q = 0; q < n_bgroups; ++q) {
            a.grp_base = q;
            CK(launch_adjoint_faces<F>(a, grid, block, ctx->st));
            ctx->launches += 1;
        }
    } else {
        CK(launch_adjoint<F>(a, grid, block, ctx->st));
        ctx->launches += 1;
    }
    CK(cudaEventRecord(ctx->ev_stop[TT_STATS_ADJOINT], ctx->st));
    ctx->stats[TT_STATS_ADJOINT].grid_blocks = grid;
    ctx->stats[TT_STATS_ADJOINT].block_threads = block;
    tt_status r = finish_solve(ctx, B, h_iters, o->max_iter_adj, "tt_adjoint", TT_STATS_ADJOINT);
    if (r == TT_OK && ctx->h_pinned[2 * TT_MAX_BATCH + 1] == 0) {
        int *h = ctx->h_pinned + 2 * TT_MAX_BATCH + 2;
        CK(cudaMemcpy(h, (int *)ctx->flags.p + 2, sizeof(int), cudaMemcpyDeviceToHost));
        if (*h) return fail(ctx, TT_EINVAL, "tt_adjoint: receiver outside the grid");
    }
    return r;
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
}

const char *tt_last_error(const tt_ctx *ctx) { return ctx ? ctx->err : "no context"; }

tt_status tt_ctx_create(tt_ctx **out, const tt_grid *grid, void *cuda_stream) {
    if (!out || !grid) return TT_EINVAL;
    *out = nullptr;
    const tt_grid &G = *grid;
    int dims[3] = {G.n_r, G.n_t, G.n_p};
    for (int d : dims)
        if (d < 4 || d > TT_MAX_DIM) return TT_EINVAL;
    if (!(G.depth_max_km > G.depth_min_km) || !(G.lat_max_deg > G.lat_min_deg) ||
        !(G.lon_max_deg > G.lon_min_deg) || !(G.earth_radius_km > G.depth_max_km))
        return TT_EINVAL;
    if (G.geometry != TT_GEOM_SPHERICAL && G.geometry != TT_GEOM_FLAT) return TT_EINVAL;
    if (G.geometry == TT_GEOM_SPHERICAL &&
        (G.lat_min_deg <= -89.0 || G.lat_max_deg >= 89.0))
        return TT_EINVAL;
    tt_ctx *ctx = new tt_ctx();
    ctx->grid = G;
    ctx->st = (cudaStream_t)cuda_stream;
    const double deg = 3.14159265358979323846 / 180.0;
    GridC &g = ctx->g;
    g.nr = G.n_r; g.nt = G.n_t; g.np = G.n_p;
    g.flat = G.geometry == TT_GEOM_FLAT;
    g.N = (long long)g.nr * g.nt * g.np;
    g.re = G.earth_radius_km;
    g.r0 = G.earth_radius_km - G.depth_max_km;
    g.dr = (G.depth_max_km - G.depth_min_km) / (g.nr - 1);
    g.t0 = G.lat_min_deg * deg;
    g.dt = (G.lat_max_deg - G.lat_min_deg) * deg / (g.nt - 1);
    g.p0 = G.lon_min_deg * deg;
    g.dp = (G.lon_max_deg - G.lon_min_deg) * deg / (g.np - 1);
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
            cudaEventCreate(&ctx->ev_stop[q]) != cudaSuccess)
            s = fail(ctx, TT_ECUDA, "cudaEventCreate failed");
    if (s == TT_OK && cudaMallocHost((void **)&ctx->h_pinned,
                                     sizeof(int) * (2 * TT_MAX_BATCH + 8) +
                                         sizeof(BarrierState) * kMaxBarrierGroups) != cudaSuccess)
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
    DevBuf *bufs[] = {&ctx->src, &ctx->pts, &ctx->tabT, &ctx->tabP, &ctx->rec, &ctx->partial,
                      &ctx->conv, &ctx->iters, &ctx->nact, &ctx->bar, &ctx->flags, &ctx->cq,
                      &ctx->wq, &ctx->sidx, &ctx->next, &ctx->heads, &ctx->nheads, &ctx->JS,
                      &ctx->coef, &ctx->t0c};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    for (int q = 0; q < 2; ++q) {
        if (ctx->ev_start[q]) cudaEventDestroy(ctx->ev_start[q]);
        if (ctx->ev_stop[q]) cudaEventDestroy(ctx->ev_stop[q]);
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
    if (!d || !d_T || !d_R || !d->d_abs_off || !d->d_cs_off)
        return fail(ctx, TT_EINVAL, "tt_misfit: NULL argument");
    if (dtype != TT_F32 && dtype != TT_F64) return fail(ctx, TT_EINVAL, "bad dtype %d", dtype);
    if (d->n_src < 1 || d->n_src > TT_MAX_BATCH)
        return fail(ctx, TT_EINVAL, "n_src = %d outside 1..%d", d->n_src, TT_MAX_BATCH);
    if ((size_t)d->n_rec * 2 * 4 * sizeof(double) > 200 * 1024)
        return fail(ctx, TT_EINVAL, "n_rec = %d too large for the misfit kernel", d->n_rec);
    tt_status s;
    ENSURE(ctx->flags, 4 * sizeof(int));
    CK(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), ctx->st));
    if ((s = receivers_impl(ctx, d->h_rec, d->n_rec)) != TT_OK) return s;
    int *bad = (int *)ctx->flags.p + 1;
    if (dtype == TT_F32)
        CK(run_misfit<float>(d->n_src, d->n_rec, d_T, (const long long *)ctx->cq.p,
                             (const double *)ctx->wq.p, *d, d_Tr, d_chi, d_R, bad, ctx->st));
    else
        CK(run_misfit<double>(d->n_src, d->n_rec, d_T, (const long long *)ctx->cq.p,
                              (const double *)ctx->wq.p, *d, d_Tr, d_chi, d_R, bad, ctx->st));
    ctx->launches += 1;
    int *h = ctx->h_pinned + 2 * TT_MAX_BATCH + 4;
    CK(cudaMemcpyAsync(h, (int *)ctx->flags.p + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h[0]) return fail(ctx, TT_EINVAL, "tt_misfit: receiver index out of range in the data");
    if (h[1]) return fail(ctx, TT_EINVAL, "tt_misfit: receiver outside the grid");
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
    if (model->dtype == TT_F32)
        CK(run_kernel_accum<float>(ctx->g, n_src, model->d_s, d_T, d_P, ctx->gd.h2, ctx->gd.cost,
                                   d_Ks, d_Kxi, d_Keta, ctx->n_sm, ctx->st));
    else
        CK(run_kernel_accum<double>(ctx->g, n_src, model->d_s, d_T, d_P, ctx->gd.h2,
                                    ctx->gd.cost, d_Ks, d_Kxi, d_Keta, ctx->n_sm, ctx->st));
    ctx->launches += 1;
    return TT_OK;
}

tt_status tt_get_stats(const tt_ctx *ctx, int which, tt_stats *out) {
    if (!ctx || !out || (which != TT_STATS_FORWARD && which != TT_STATS_ADJOINT))
        return TT_EINVAL;
    *out = ctx->stats[which];
    out->launches = ctx->launches;
    return TT_OK;
}

}  // extern "C"
