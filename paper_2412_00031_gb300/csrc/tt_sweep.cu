// Persistent fast-sweeping kernels of libttgb: the factored Lax-Friedrichs forward sweep
// (Eq. "4", Sec. 3.1) and the upwind adjoint sweep (Eq. 5), both run hyperplane by
// hyperplane (Sec. 3.4) inside one cooperative launch per solve.
//
// Work mapping. Batched fields are stored [node][source]. Thread t of the launch owns one
// source b = t mod B for the whole solve and a slot t / B; on each hyperplane the slots
// stride over the plane's nodes. With B >= 32 a warp reads 32 consecutive sources of one
// node, so every field access is a coalesced 128-byte line and the per-node model values
// are warp-wide broadcasts. Between hyperplanes the launch crosses a bounded grid barrier.
#include <cuda.h>
#include <cuda_runtime.h>

#include "tt_internal.h"

namespace ttgb {

template <typename F> __device__ __forceinline__ F fmax_(F a, F b) { return a > b ? a : b; }

__device__ __forceinline__ void atomic_max_nonneg(float *p, float v) {
    atomicMax(reinterpret_cast<unsigned int *>(p), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double *p, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(p),
              (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void unpack(unsigned int pk, int &a, int &b, int &c) {
    a = (int)(pk >> 20);
    b = (int)((pk >> 10) & 1023u);
    c = (int)(pk & 1023u);
}

// ------------------------------------------------------------------------ forward sweep

// Factor cache: 1/T0 and u = grad T0 / T0 (factor_T0) of every (node, source) of a launch,
// computed once per solve; 1/T0 = -1 marks the nodes of the source's fixed set. Every schedule reads the same cached values, so every schedule
// performs exactly the same arithmetic.
template <typename F> __global__ void t0_cache_kernel(FwdArgs<F> a) {
    const GridC &g = a.g;
    const long long total = g.N * a.src_n;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const int bl = (int)(x % a.src_n);
        const int b = a.src_lo + bl;
        const long long n = x / a.src_n;
        const int k = (int)(n % g.np);
        const long long t = n / g.np;
        const int j = (int)(t % g.nt), i = (int)(t / g.nt);
        const SrcReg<F> S = load_src<F>(a.src, b, g.dr);
        Vec4<F> c;
        c.x = factor_T0<F>(S, i, __ldg(a.rad + i), __ldg(a.cost + j), __ldg(a.sint + j),
                           a.tabT[(long long)j * a.B + b], a.tabP[(long long)k * a.B + b],
                           g.flat != 0, c.y, c.z, c.w);
        // nodes of the fixed set are never swept: mark them with 1/T0 = -1
        if (in_fixed_set(S.ci, S.cj, S.ck, i, j, k)) c.x = (F)-1;
        a.t0c[x] = c;
    }
}

// tau on one face layer = max(2 tau_1 - tau_2, tau_2); q enumerates both faces of an axis.
template <typename F>
__device__ __forceinline__ void extrapolate(const FwdArgs<F> &a, int b, int axis, int slot,
                                            int slots) {
    const GridC &g = a.g;
    const int ci = a.src[b].ci, cj = a.src[b].cj, ck = a.src[b].ck;  // fixed set centre
    const long long B = a.B;
    int n1, n2, nface;
    long long stride;
    if (axis == 0) { n1 = g.nt; n2 = g.np; nface = g.nr; stride = (long long)g.nt * g.np; }
    else if (axis == 1) { n1 = g.nr; n2 = g.np; nface = g.nt; stride = g.np; }
    else { n1 = g.nr; n2 = g.nt; nface = g.np; stride = 1; }
    const int per_face = n1 * n2;
    for (int q = slot; q < 2 * per_face; q += slots) {
        int hi = q >= per_face;
        int rem = hi ? q - per_face : q;
        int u = rem / n2, v = rem - u * n2;
        int f0 = hi ? nface - 1 : 0, f1 = hi ? nface - 2 : 1, f2 = hi ? nface - 3 : 2;
        int i, j, k;
        if (axis == 0) { i = f0; j = u; k = v; }
        else if (axis == 1) { i = u; j = f0; k = v; }
        else { i = u; j = v; k = f0; }
        if (in_fixed_set(ci, cj, ck, i, j, k)) continue;
        long long n = node_index(g, i, j, k);
        long long x0 = n * B + b;
        long long x1 = x0 + (long long)(f1 - f0) * stride * B;
        long long x2 = x0 + (long long)(f2 - f0) * stride * B;
        F t1 = a.tau[x1], t2 = a.tau[x2];
        a.tau[x0] = fmax_((F)2 * t1 - t2, t2);
    }
}

// The same extrapolation for all NS sources of a lane (b + 32 h, those with act[h]): the
// loads of all of them are issued before the stores (K face nodes at a time; more than one
// costs the sweep kernel registers). Within one axis the
// written layer (0 or n - 1) is never a layer read (1, 2 or n - 2, n - 3; n >= 4), so the
// order of the face nodes does not matter and the bits equal extrapolate()'s.
template <typename F, int NS>
__device__ __forceinline__ void extrapolate_lane(const FwdArgs<F> &a, int b, const bool (&act)[NS],
                                                 int axis, int slot, int slots) {
    constexpr int K = 1;
    const GridC &g = a.g;
    const long long B = a.B;
    int n1, n2, nface;
    long long stride;
    if (axis == 0) { n1 = g.nt; n2 = g.np; nface = g.nr; stride = (long long)g.nt * g.np; }
    else if (axis == 1) { n1 = g.nr; n2 = g.np; nface = g.nt; stride = g.np; }
    else { n1 = g.nr; n2 = g.nt; nface = g.np; stride = 1; }
    const long long sB = stride * B;   // one layer inwards from the low face
    const int per_face = n1 * n2;
    for (int q0 = slot; q0 < 2 * per_face; q0 += K * slots) {
        long long x0[K];
        int ii[K], jj[K], kk[K];
        bool okq[K], hiq[K];
        F t1[K][NS], t2[K][NS];
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const int q = q0 + u * slots;
            okq[u] = q < 2 * per_face;
            hiq[u] = q >= per_face;
            const int rem = okq[u] ? (hiq[u] ? q - per_face : q) : 0;
            const int uu = rem / n2, vv = rem - uu * n2;
            const int f0 = hiq[u] ? nface - 1 : 0;
            if (axis == 0) { ii[u] = f0; jj[u] = uu; kk[u] = vv; }
            else if (axis == 1) { ii[u] = uu; jj[u] = f0; kk[u] = vv; }
            else { ii[u] = uu; jj[u] = vv; kk[u] = f0; }
            x0[u] = node_index(g, ii[u], jj[u], kk[u]) * B + b;
            const long long d = hiq[u] ? -sB : sB;
#pragma unroll
            for (int h = 0; h < NS; ++h)
                if (okq[u] && act[h]) {
                    t1[u][h] = a.tau[x0[u] + d + 32 * h];
                    t2[u][h] = a.tau[x0[u] + 2 * d + 32 * h];
                }
        }
#pragma unroll
        for (int u = 0; u < K; ++u)
#pragma unroll
            for (int h = 0; h < NS; ++h) {
                if (!(okq[u] && act[h])) continue;
                const SrcC &sc = a.src[b + 32 * h];
                if (!in_fixed_set(sc.ci, sc.cj, sc.ck, ii[u], jj[u], kk[u]))
                    a.tau[x0[u] + 32 * h] = fmax_((F)2 * t1[u][h] - t2[u][h], t2[u][h]);
            }
    }
}

// Retire-and-refill: for every slot x of a group whose fill flag is set, copy the
// retiring source's column of tau to the output and load the new source into the slot:
// tau = 1 (or the caller's tau), the fixed set tau = 1, and its factor cache column,
// computed exactly as t0_cache_kernel does. The group's threads stride over the nodes.
template <typename F>
__device__ void refill_slots(const FwdArgs<F> &a, int src0, int Bg, int blk) {
    const GridC &g = a.g;
    const long long S = a.B, NA = a.n_all;
    const long long stride = (long long)a.grp_blocks * blockDim.x;
    const long long first = (long long)blk * blockDim.x + threadIdx.x;
    for (int x = src0; x < src0 + Bg; ++x) {
        if (((volatile int *)a.slot_fill)[x] == 0) continue;
        const int old = ((volatile int *)a.slot_prev)[x], nw = ((volatile int *)a.slot_src)[x];
        SrcReg<F> S_;
        if (nw >= 0) S_ = load_src<F>(a.src_all, nw, g.dr);
        for (long long n = first; n < g.N; n += stride) {
            const long long xs = n * S + x;
            if (old >= 0) a.tau_out[n * NA + old] = a.tau[xs];
            if (nw < 0) continue;
            const int k = (int)(n % g.np);
            const long long tq = n / g.np;
            const int j = (int)(tq % g.nt), i = (int)(tq / g.nt);
            Vec4<F> c;
            c.x = factor_T0<F>(S_, i, __ldg(a.rad + i), __ldg(a.cost + j), __ldg(a.sint + j),
                               a.tabT_all[(long long)j * NA + nw], a.tabP_all[(long long)k * NA + nw],
                               g.flat != 0, c.y, c.z, c.w);
            const bool fixed = in_fixed_set(S_.ci, S_.cj, S_.ck, i, j, k);
            if (fixed) c.x = (F)-1;
            a.t0c[xs] = c;
            a.tau[xs] = fixed || !a.init_from_out ? (F)1 : a.tau_out[n * NA + nw];
        }
    }
}

template <typename F> __global__ void refill_setup_kernel(FwdArgs<F> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x == 0) *a.queue = a.B < a.n_all ? a.B : a.n_all;
    if (x >= a.B) return;
    const bool has = x < a.n_all;
    a.slot_src[x] = has ? x : -1;
    a.slot_prev[x] = -1;
    a.slot_it[x] = 0;
    a.slot_fill[x] = has ? 1 : 0;
    if (has) a.slot_srcc[x] = a.src_all[x];
}

// Node-hyperplane schedule. The launch is split into barrier groups: group g owns a
// contiguous slice of the launch's sources and a contiguous range of blocks, runs the whole
// solve of its slice with its own grid barrier and convergence test, and so never waits for
// another group; on each SM the warps of one group keep issuing while another group's warps
// wait at their barrier.
//
// Within a group, a warp covers 64 consecutive sources of one node: lane l holds sources
// l and l + 32 of its 64, so both of a lane's accesses are coalesced 128-byte lines and the
// second is the first plus a constant offset. A slot is the set of warps that cover the
// group's sources (padded to whole warps); on a hyperplane each slot takes the nodes slot,
// slot + slots, ... The schedule is static, so the index of a thread's next node, the
// bounds of the next hyperplane and the index of its first node there are read one step
// ahead (the latter two before the barrier), off the critical path. The node record (8
// values shared by the warp) is read by every lane as two broadcast 16-byte loads. The
// factor cache is read once per sweep and streamed past L2 (evict-first), so that it does
// not push out the tau lines the next hyperplane reads.
#ifndef TTGB_FWD_MIN_BLOCKS
#define TTGB_FWD_MIN_BLOCKS 4
#endif
// The Godunov updates do several times the arithmetic of Lax-Friedrichs per node; their
// instantiations get a larger register budget (fewer resident blocks per SM).
#ifndef TTGB_GOD_MIN_BLOCKS
#define TTGB_GOD_MIN_BLOCKS 3
#endif

// Sweep-local node (aa, bb, cc) -> offset of its node index from the sweep's first node.
template <typename I>
__device__ __forceinline__ I node_local(unsigned pk, I sa, I sb, I sc) {
    int aa, bb, cc;
    unpack(pk, aa, bb, cc);
    return (I)aa * sa + (I)bb * sb + (I)cc * sc;
}

// The node record read by every lane as broadcast vector loads (one 16-byte request per
// half, served to the whole warp).
__device__ __forceinline__ NodeRec<float> rec_vec(const NodeRec<float> *r) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(r));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(r) + 1);
    NodeRec<float> R;
    R.s = a.x; R.xi = a.y; R.eta = a.z; R.ct = a.w;
    R.cp = b.x; R.invW = b.y; R.et = b.z; R.ep = b.w;
    return R;
}
__device__ __forceinline__ NodeRec<double> rec_vec(const NodeRec<double> *r) {
    const double2 *q = reinterpret_cast<const double2 *>(r);
    const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
    NodeRec<double> R;
    R.s = a.x; R.xi = a.y; R.eta = b.x; R.ct = b.y;
    R.cp = c.x; R.invW = c.y; R.et = d.x; R.ep = d.y;
    return R;
}

__device__ __forceinline__ Vec4<float> ld_stream(const Vec4<float> *p) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    return Vec4<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Vec4<double> ld_stream(const Vec4<double> *p) {
    const double2 v0 = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 v1 = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    return Vec4<double>{v0.x, v0.y, v1.x, v1.y};
}

// Lax-Friedrichs update of one (node, source): tau at p, its six neighbours at p +- sr,
// p +- st, p +- sp; c = the cached factors. Returns |change| (0 on the fixed set).
__device__ __forceinline__ unsigned bits_of(float x) { return __float_as_uint(x); }
__device__ __forceinline__ unsigned long long bits_of(double x) {
    return (unsigned long long)__double_as_longlong(x);
}

template <typename F, int SCHEME>
__device__ __forceinline__ F update_one(F *p, const F *v, const Vec4<F> &c, const NodeRec<F> &R,
                                        F er) {
    if (!(c.x > (F)0)) return (F)0;
    const F tn =
        SCHEME == 2   ? godunov_aniso_core<F>(c.x, c.y, c.z, c.w, v[0], v[1], v[2], v[3], v[4], v[5], v[6], R, er)
        : SCHEME == 1 ? godunov_core<F>(c.x, c.y, c.z, c.w, v[0], v[1], v[2], v[3], v[4], v[5], v[6], R, er)
                      : lf_core<F>(c.x, c.y, c.z, c.w, v[0], v[1], v[2], v[3], v[4], v[5], v[6], R, er);
    // a value that keeps its bits is not stored, so that its line is not made dirty (late
    // in a solve most values have stopped changing)
    if (bits_of(tn) != bits_of(v[0])) *p = tn;
    return fabs(tn - v[0]);
}

// I: index type of the [node][source] fields (32-bit when every index fits).
// REFILL: the retire-and-refill mode (compiled separately, so that the resident launch
// carries none of its code). SCHEME: the local solver, 0 Lax-Friedrichs (lf_core), 1 Godunov
// (godunov_core, isotropic models), 2 Godunov for anisotropic models (godunov_aniso_core),
// 3 Lax-Friedrichs on T itself with the faces held fixed (the region's solve of teleseismic
// events: lf_core with T0 = 1 and no factor gradient, no factor cache read, no fixed set,
// no face extrapolation; the "sources" are the events).
template <typename F, typename I, bool REFILL, int SCHEME>
__global__ void __launch_bounds__(256, (SCHEME == 0 || SCHEME == 3) ? TTGB_FWD_MIN_BLOCKS
                                                                    : TTGB_GOD_MIN_BLOCKS)
    fwd_sweep_kernel(FwdArgs<F> a) {
    constexpr int NS = kFwdSourcesPerLane;              // sources of one lane: l0 + 32 h
    extern __shared__ unsigned char smem_raw[];
    F *s_err = reinterpret_cast<F *>(smem_raw);
    __shared__ int s_cnt;
    const GridC &g = a.g;
    const int B = a.B;
    const int grp = blockIdx.x / a.grp_blocks;
    const int blk = blockIdx.x - grp * a.grp_blocks;   // block index within the group
    const int src0 = a.src_lo + grp * a.grp_src;
    const int Bg = min(a.src_lo + a.src_n, src0 + a.grp_src) - src0;  // sources of the group
    if (Bg <= 0) return;
    barrier_begin();
    const int Bw = (Bg + 32 * NS - 1) / (32 * NS) * 32; // lanes of one slot
    BarrierState *bar = a.bar + grp;
    const unsigned nblk = (unsigned)a.grp_blocks;
    const int slots = (int)(((long long)a.grp_blocks * blockDim.x) / Bw);
    const long long tid = (long long)blk * blockDim.x + threadIdx.x;
    const bool lane_ok = tid < (long long)slots * Bw;   // uniform over a warp
    const int bl = lane_ok ? (int)(tid % Bw) : 0;
    const int slot = lane_ok ? (int)(tid / Bw) : 0;
    const int lane = threadIdx.x & 31;
    const int l0 = (bl >> 5) * (32 * NS) + lane;        // the lane's first source in the group
    bool okh[NS];
#pragma unroll
    for (int h = 0; h < NS; ++h) okh[h] = lane_ok && l0 + 32 * h < Bg;
    const int b = src0 + (okh[0] ? l0 : 0);             // the lane's sources: b + 32 h
    const I sp = (I)B, st = (I)g.np * (I)B, sr = (I)g.nt * (I)g.np * (I)B;
    const long long osr = (long long)sr, ost = (long long)st, osp = (long long)sp;  // signed
    const I snode_r = (I)g.nt * (I)g.np, snode_t = (I)g.np;
    const Vec4<F> *t0c = a.t0c + (b - a.src_lo);
    const I src_n = (I)a.src_n;
    F *tau = a.tau;

    // retire-and-refill: load the group's first sources into their slots
    if (REFILL) {
        refill_slots<F>(a, src0, Bg, blk);
        if (!grid_barrier(bar, a.spin_ns, nblk)) return;
    }
    // with refill a group runs until its queue is empty; each source still stops at max_iter
    const long long it_end = REFILL ? (long long)a.max_iter * (a.n_all + 1) : a.max_iter;
    for (long long it = 0; it < it_end; ++it) {
        bool act[NS];
        bool any = false;
#pragma unroll
        for (int h = 0; h < NS; ++h) {
            act[h] = okh[h] && (REFILL ? ((volatile int *)a.slot_src)[b + 32 * h] >= 0
                                       : ((volatile int *)a.conv)[b + 32 * h] == 0);
            any = any || act[h];
        }
        const bool busy = lane_ok && __any_sync(0xffffffffu, any);  // uniform
        F err[NS];
#pragma unroll
        for (int h = 0; h < NS; ++h) err[h] = 0;
        for (int o = 0; o < 8; ++o) {
            const bool rr = o & 4, rt = o & 2, rp = o & 1;
            // node index of sweep-local (aa, bb, cc): n0 + aa * sa + bb * sb + cc * sc
            const I n0 = (I)(rr ? g.nr - 2 : 1) * snode_r + (I)(rt ? g.nt - 2 : 1) * snode_t +
                         (I)(rp ? g.np - 2 : 1);
            const I sa = rr ? (I)0 - snode_r : snode_r, sb = rt ? (I)0 - snode_t : snode_t;
            const I sc = rp ? (I)0 - (I)1 : (I)1;
            // this thread's nodes of plane L: q = qa, qa + slots, ... < qe; pk = index of qa
            int qa = __ldg(a.off) + slot, qe = __ldg(a.off + 1);
            unsigned pk = busy && qa < qe ? __ldg(a.nodes + qa) : 0u;
            for (int L = 0; L < a.n_planes; ++L) {
                const bool last = L + 1 == a.n_planes;
                const int qe_next = last ? 0 : __ldg(a.off + L + 2);
                if (busy) {
                    for (int q = qa; q < qe; q += slots) {
                        const int qn = q + slots;
                        const unsigned pkn = qn < qe ? __ldg(a.nodes + qn) : 0u;
                        const I n = n0 + node_local(pk, sa, sb, sc);
                        F *p = tau + (n * (I)B + (I)b);
                        const Vec4<F> *pc = t0c + n * src_n;
                        F v[NS][7];
                        Vec4<F> c[NS];
#pragma unroll
                        for (int h = 0; h < NS; ++h) {
                            if (!act[h]) continue;
                            const F *ph = p + 32 * h;
                            v[h][0] = ph[0];
                            v[h][1] = ph[osr];
                            v[h][2] = ph[-osr];
                            v[h][3] = ph[ost];
                            v[h][4] = ph[-ost];
                            v[h][5] = ph[osp];
                            v[h][6] = ph[-osp];
                            c[h] = SCHEME == 3 ? Vec4<F>{(F)1, (F)0, (F)0, (F)0}
                                               : ld_stream(pc + 32 * h);
                        }
                        const NodeRec<F> R = rec_vec(a.rec + n);
#pragma unroll
                        for (int h = 0; h < NS; ++h)
                            if (act[h])
                                err[h] = fmax_(err[h], update_one<F, SCHEME>(p + 32 * h, v[h], c[h], R, a.er));
                        pk = pkn;
                    }
                }
                // first node of the next plane (static: needs no barrier)
                const int qa_next = qe + slot;
                if (busy && !last && qa_next < qe_next) pk = __ldg(a.nodes + qa_next);
                if (!grid_barrier(bar, a.spin_ns, nblk)) return;
                qa = qa_next;
                qe = qe_next;
            }
            if (SCHEME != 3)  // SCHEME 3 holds the faces fixed
                for (int axis = 0; axis < 3; ++axis) {
                    if (any) extrapolate_lane<F, NS>(a, b, act, axis, slot, slots);
                    if (!grid_barrier(bar, a.spin_ns, nblk)) return;
                }
        }
        // Per-source largest update of this iteration: block maximum, then a fixed-order
        // maximum over the group's blocks by its first block, which also decides convergence.
        for (int x = threadIdx.x; x < Bg; x += blockDim.x) s_err[x] = 0;
        __syncthreads();
#pragma unroll
        for (int h = 0; h < NS; ++h)
            if (act[h]) atomic_max_nonneg(&s_err[b + 32 * h - src0], err[h]);
        __syncthreads();
        for (int x = threadIdx.x; x < Bg; x += blockDim.x)
            a.partial[(long long)blockIdx.x * B + src0 + x] = s_err[x];
        if (!grid_barrier(bar, a.spin_ns, nblk)) return;
        if (blk == 0) {
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            for (int x = src0 + threadIdx.x; x < src0 + Bg; x += blockDim.x) {
                if (REFILL) {
                    // slots: a finished source hands its slot to the next queued source
                    a.slot_fill[x] = 0;
                    const int s = a.slot_src[x];
                    if (s < 0) continue;
                    F m = 0;
                    for (int c = grp * a.grp_blocks; c < (grp + 1) * a.grp_blocks; ++c)
                        m = fmax_(m, ((volatile F *)a.partial)[(long long)c * B + x]);
                    const int its = a.slot_it[x] + 1;
                    a.slot_it[x] = its;
                    if (!(m < a.tol) && its < a.max_iter) {
                        atomicAdd(&s_cnt, 1);
                        continue;
                    }
                    a.iters[s] = its;
                    a.conv[s] = m < a.tol ? 1 : 0;
                    const int nw = atomicAdd(a.queue, 1);
                    a.slot_prev[x] = s;
                    a.slot_fill[x] = 1;
                    a.slot_it[x] = 0;
                    if (nw < a.n_all) {
                        a.slot_src[x] = nw;
                        a.slot_srcc[x] = a.src_all[nw];
                        atomicAdd(&s_cnt, 1);
                    } else {
                        a.slot_src[x] = -1;
                    }
                    continue;
                }
                if (a.conv[x]) continue;
                F m = 0;
                for (int c = grp * a.grp_blocks; c < (grp + 1) * a.grp_blocks; ++c)
                    m = fmax_(m, ((volatile F *)a.partial)[(long long)c * B + x]);
                a.iters[x] = (int)it + 1;
                if (m < a.tol) a.conv[x] = 1;
                else atomicAdd(&s_cnt, 1);
            }
            __syncthreads();
            if (threadIdx.x == 0) ((volatile int *)a.n_active)[grp] = s_cnt;
        }
        if (!grid_barrier(bar, a.spin_ns, nblk)) return;
        if (REFILL) {
            // retire the finished columns and load the new sources, then start them together
            refill_slots<F>(a, src0, Bg, blk);
            if (!grid_barrier(bar, a.spin_ns, nblk)) return;
        }
        if (((volatile int *)a.n_active)[grp] == 0) break;
    }
    barrier_end(bar, nblk);
}

// ------------------------------------------------------------------------ tiled forward sweep
//
// Tile wavefront (Sec. 3.4 applied to tiles). The interior swept by one ordering is cut into
// TA x TB x TC tiles in sweep-local coordinates; tiles with the same I + J + K share no
// face, so they run concurrently, and one bounded grid barrier separates consecutive tile
// hyperplanes. A block task is (tile, group of 32 sources). One thread issues two TMA
// tensor copies: the tile with a one-node halo of tau for those 32 sources (a 4-D box
// sources x phi x theta x r of the [node][source] field) and the tile's per-node records.
// The box lands in shared memory in physical order, so the six neighbours of a node are at
// fixed offsets. The block then runs the tile's node hyperplanes in sweep order with block
// barriers (every node sees exactly the neighbour values of the lexicographic sweep) and
// writes the tile back with coalesced 128-byte stores (lanes = sources).


__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bounded wait on an mbarrier phase; false when the limit expired.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          unsigned long long limit_ns) {
    const unsigned sa = smem_u32(bar);
    unsigned long long t0 = 0;
    for (int spin = 0;; ++spin) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(sa), "r"(parity)
            : "memory");
        if (ok) return true;
        if (spin == 0) t0 = global_ns();
        else if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int TA, int TB, int TC> struct TileDims {
    static constexpr int HA = TA + 2, HB = TB + 2, HC = TC + 2;
    static constexpr int ROWS = HA * HB * HC;              // halo'd nodes staged per task
    static constexpr int NODES = TA * TB * TC;
    static constexpr int PLANES = TA + TB + TC - 2;
    static constexpr int SA = HB * HC * 32, SB = HC * 32;  // smem strides (elements)
};

template <typename F, int TA, int TB, int TC> struct TileSmem {
    using D = TileDims<TA, TB, TC>;
    static constexpr size_t tau = 0;
    static constexpr size_t rec = tau + sizeof(F) * D::ROWS * 32;
    static constexpr size_t cache = rec + sizeof(NodeRec<F>) * D::NODES;
    static constexpr size_t plist = cache + sizeof(Vec4<F>) * D::NODES * 32;
    static constexpr size_t poff = plist + sizeof(unsigned short) * D::NODES;
    static constexpr size_t err = (poff + sizeof(int) * (D::PLANES + 1) + 15) / 16 * 16;
    static_assert(rec % 128 == 0 && cache % 128 == 0, "TMA destinations need 128-byte alignment");
};

template <typename F, int TA, int TB, int TC>
__device__ __forceinline__ bool forward_tile(const FwdArgs<F> &a, const CUtensorMap *map_tau,
                                             const CUtensorMap *map_rec,
                                             const CUtensorMap *map_t0c, int I, int J, int K,
                                             int grp, bool rr, bool rt, bool rp,
                                             unsigned char *smem, unsigned long long *bar,
                                             unsigned &parity, F *s_err) {
    using D = TileDims<TA, TB, TC>;
    using L = TileSmem<F, TA, TB, TC>;
    F *s_tau = reinterpret_cast<F *>(smem + L::tau);
    const NodeRec<F> *s_rec = reinterpret_cast<const NodeRec<F> *>(smem + L::rec);
    const Vec4<F> *s_t0c = reinterpret_cast<const Vec4<F> *>(smem + L::cache);
    const unsigned short *s_plist = reinterpret_cast<const unsigned short *>(smem + L::plist);
    const int *s_poff = reinterpret_cast<const int *>(smem + L::poff);
    const GridC &g = a.g;
    const int B = a.B;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int a0 = I * TA, b0 = J * TB, c0 = K * TC;
    // physical index of the tile's first interior node on each axis (lowest index)
    const int i_lo = rr ? g.nr - 1 - a0 - TA : 1 + a0;
    const int j_lo = rt ? g.nt - 1 - b0 - TB : 1 + b0;
    const int k_lo = rp ? g.np - 1 - c0 - TC : 1 + c0;

    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(bar, (unsigned)(sizeof(F) * (D::ROWS * 32 + D::NODES * (8 + 128))));
        tma_load_4d(s_tau, map_tau, a.src_lo + grp * 32, k_lo - 1, j_lo - 1, i_lo - 1, bar);
        tma_load_4d(smem + L::rec, map_rec, 0, k_lo, j_lo, i_lo, bar);
        tma_load_4d(smem + L::cache, map_t0c, grp * 128, k_lo, j_lo, i_lo, bar);
    }
    const int bsrc = a.src_lo + grp * 32 + lane;
    const bool valid = bsrc < a.src_lo + a.src_n;
    const bool active = valid && ((volatile int *)a.conv)[bsrc] == 0;
    const SrcReg<F> S = load_src<F>(a.src, valid ? bsrc : a.src_lo, g.dr);
    const bool landed = mbar_wait(bar, parity, a.spin_ns);
    if (!landed) {
        // record the failure, then give the copies in flight one more bounded wait before
        // this block stops using its shared memory
        atomicExch(&a.bar->status, (int)kDevTimeout);
        mbar_wait(bar, parity, a.spin_ns);
    }
    parity ^= 1u;
    __syncthreads();
    if (ld_status(&a.bar->status) != 0) return false;

    F err = 0;
    for (int l = 0; l < D::PLANES; ++l) {
        for (int e = s_poff[l] + warp; e < s_poff[l + 1]; e += nwarps) {
            const unsigned pk = s_plist[e];
            const int ta = pk >> 10, tb = (pk >> 5) & 31, tc = pk & 31;
            const int la = a0 + ta, lb = b0 + tb, lc = c0 + tc;
            if (la >= a.na || lb >= a.nb || lc >= a.nc) continue;
            const int i = rr ? g.nr - 2 - la : 1 + la;
            const int j = rt ? g.nt - 2 - lb : 1 + lb;
            const int k = rp ? g.np - 2 - lc : 1 + lc;
            if (!active || in_fixed_set(S.ci, S.cj, S.ck, i, j, k)) continue;
            const int pa = i - i_lo + 1, pb = j - j_lo + 1, pc = k - k_lo + 1;
            F *p = s_tau + ((pa * D::HB + pb) * D::HC + pc) * 32 + lane;
            const F t0 = p[0];
            const int nl = ((pa - 1) * TB + (pb - 1)) * TC + (pc - 1);
            const NodeRec<F> R = s_rec[nl];
            const Vec4<F> c = s_t0c[nl * 32 + lane];
            const F tn = lf_core<F>(c.x, c.y, c.z, c.w, t0, p[D::SA], p[-D::SA], p[D::SB],
                                    p[-D::SB], p[32], p[-32], R, a.er);
            p[0] = tn;
            err = fmax_(err, fabs(tn - t0));
        }
        __syncthreads();
    }

    // write the tile back (only sources that are still iterating changed anything)
    if (active) {
        for (int e = warp; e < D::NODES; e += nwarps) {
            const int qa = e / (TB * TC), rem = e - qa * (TB * TC);
            const int qb = rem / TC, qc = rem - qb * TC;
            const int i = i_lo + qa, j = j_lo + qb, k = k_lo + qc;
            if (i < 1 || j < 1 || k < 1 || i > g.nr - 2 || j > g.nt - 2 || k > g.np - 2) continue;
            a.tau[node_index(g, i, j, k) * B + bsrc] =
                s_tau[(((qa + 1) * D::HB + (qb + 1)) * D::HC + (qc + 1)) * 32 + lane];
        }
        atomic_max_nonneg(&s_err[bsrc], err);
    }
    __syncthreads();
    return true;
}

template <typename F, int TA, int TB, int TC>
__global__ void __launch_bounds__(kTileThreads)
    fwd_tile_kernel(const __grid_constant__ CUtensorMap map_tau,
                    const __grid_constant__ CUtensorMap map_rec,
                    const __grid_constant__ CUtensorMap map_t0c, FwdArgs<F> a) {
    using D = TileDims<TA, TB, TC>;
    using L = TileSmem<F, TA, TB, TC>;
    extern __shared__ __align__(1024) unsigned char smem[];
    F *s_err = reinterpret_cast<F *>(smem + L::err);
    int *s_gact = reinterpret_cast<int *>(s_err + a.B);
    __shared__ int s_cnt;
    __shared__ __align__(8) unsigned long long bar;
    const GridC &g = a.g;
    const int B = a.B;
    // per-plane node lists of one tile, in sweep-local coordinates (ta << 10 | tb << 5 | tc)
    if (threadIdx.x == 0) {
        unsigned short *plist = reinterpret_cast<unsigned short *>(smem + L::plist);
        int *poff = reinterpret_cast<int *>(smem + L::poff);
        int q = 0;
        for (int l = 0; l < D::PLANES; ++l) {
            poff[l] = q;
            for (int ta = 0; ta < TA; ++ta)
                for (int tb = 0; tb < TB; ++tb) {
                    const int tc = l - ta - tb;
                    if (tc >= 0 && tc < TC) plist[q++] = (unsigned short)((ta << 10) | (tb << 5) | tc);
                }
        }
        poff[D::PLANES] = q;
        mbar_init(&bar);
    }
    __syncthreads();
    unsigned parity = 0;
    // face extrapolation keeps the one-source-per-thread mapping of the node schedule
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool lane_ok = tid < (long long)a.slots * a.src_n;
    const int bx = a.src_lo + (lane_ok ? (int)(tid % a.src_n) : 0);
    const int slot = lane_ok ? (int)(tid / a.src_n) : 0;
    const int s_end = a.src_lo + a.src_n;
    barrier_begin();

    for (int it = 0; it < a.max_iter; ++it) {
        const bool act_x = lane_ok && ((volatile int *)a.conv)[bx] == 0;
        for (int x = threadIdx.x; x < B; x += blockDim.x) s_err[x] = 0;
        for (int q = threadIdx.x; q < a.ngroups; q += blockDim.x) {
            int any = 0;
            for (int x = a.src_lo + q * 32; x < min(s_end, a.src_lo + q * 32 + 32); ++x)
                any |= ((volatile int *)a.conv)[x] == 0;
            s_gact[q] = any;
        }
        __syncthreads();
        for (int o = 0; o < 8; ++o) {
            const bool rr = o & 4, rt = o & 2, rp = o & 1;
            for (int Lp = 0; Lp < a.n_tplanes; ++Lp) {
                const int t0 = __ldg(a.toff + Lp);
                const int ntask = (__ldg(a.toff + Lp + 1) - t0) * a.ngroups;
                for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
                    const int grp = task % a.ngroups;
                    if (!s_gact[grp]) continue;
                    int I, J, K;
                    unpack(__ldg(a.tiles + t0 + task / a.ngroups), I, J, K);
                    if (!forward_tile<F, TA, TB, TC>(a, &map_tau, &map_rec, &map_t0c, I, J, K,
                                                     grp, rr, rt, rp, smem, &bar, parity, s_err))
                        return;
                }
                if (!grid_barrier(a.bar, a.spin_ns)) return;
            }
            for (int axis = 0; axis < 3; ++axis) {
                if (act_x) extrapolate<F>(a, bx, axis, slot, a.slots);
                if (!grid_barrier(a.bar, a.spin_ns)) return;
            }
        }
        for (int x = threadIdx.x; x < B; x += blockDim.x)
            a.partial[(long long)blockIdx.x * B + x] = s_err[x];
        if (!grid_barrier(a.bar, a.spin_ns)) return;
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            for (int x = a.src_lo + threadIdx.x; x < s_end; x += blockDim.x) {
                if (a.conv[x]) continue;
                F m = 0;
                for (int c = 0; c < (int)gridDim.x; ++c)
                    m = fmax_(m, ((volatile F *)a.partial)[(long long)c * B + x]);
                a.iters[x] = it + 1;
                if (m < a.tol) a.conv[x] = 1;
                else atomicAdd(&s_cnt, 1);
            }
            __syncthreads();
            if (threadIdx.x == 0) *((volatile int *)a.n_active) = s_cnt;
        }
        if (!grid_barrier(a.bar, a.spin_ns)) return;
        if (*((volatile int *)a.n_active) == 0) break;
    }
    barrier_end(a.bar, gridDim.x);
}

// ------------------------------------------------------------------------ adjoint sweep

// Derivative of T along theta (axis 1) or phi (axis 2) at a node, per radian: central in
// the interior, one-sided on the faces. tm/tc/tp are T at index - 1, 0, + 1.
template <typename F>
__device__ __forceinline__ F d_axis(F tm, F tc, F tp, int idx, int n, F inv_d, F inv_2d) {
    if (idx == 0) return (tp - tc) * inv_d;
    if (idx == n - 1) return (tc - tm) * inv_d;
    return (tp - tm) * inv_2d;
}

// Upwind Gauss-Seidel update of P at node (i, j, k) for source b: the finite-volume form
// of Eq. 5 times J_c,
//   sum_d [A+ (a+^+ P_c + a+^- P_d+) - A- (a-^+ P_d- + a-^- P_c)] / delta_d = J_c S_c,
// solved for P_c, with a = -(M grad T) . n on each face (M and the cross derivative averaged
// over the face's two nodes) and no flux through the outer faces.
template <typename F>
__device__ __forceinline__ F adj_update(const AdjArgs<F> &a, int b, int i, int j, int k,
                                        long long n, F &pold) {
    const GridC &g = a.g;
    const long long B = a.B;
    const long long sp = B, st = (long long)g.np * B, sr = (long long)g.nt * g.np * B;
    const long long x = n * B + b;
    const F *T = a.T;
    const F *P = a.P;
    const bool hr = i < g.nr - 1, lr = i > 0, ht = j < g.nt - 1, lt = j > 0;
    const bool hp = k < g.np - 1, lp = k > 0;
    const F dr = (F)g.dr, dt = (F)g.dt, dp = (F)g.dp;
    const F idt = (F)1 / dt, idp = (F)1 / dp, i2dt = (F)0.5 * idt, i2dp = (F)0.5 * idp;

    const F Tc = T[x];
    const F Trp = hr ? T[x + sr] : Tc, Trm = lr ? T[x - sr] : Tc;
    const F Ttp = ht ? T[x + st] : Tc, Ttm = lt ? T[x - st] : Tc;
    const F Tpp = hp ? T[x + sp] : Tc, Tpm = lp ? T[x - sp] : Tc;
    // diagonal neighbours in the theta-phi plane (used by the cross derivatives)
    const F Tpp_tp = (ht && hp) ? T[x + st + sp] : Tc, Tpm_tp = (ht && lp) ? T[x + st - sp] : Tc;
    const F Tpp_tm = (lt && hp) ? T[x - st + sp] : Tc, Tpm_tm = (lt && lp) ? T[x - st - sp] : Tc;

    const F xic = __ldg(a.xi + n), etc = __ldg(a.eta + n);
    const F h2 = __ldg(a.h2 + i), cth = __ldg(a.cost + j);
    const F h3 = h2 * cth;

    // phi-derivatives at (j, k), (j+1, k), (j-1, k); theta-derivatives at (j, k), (j, k+1), (j, k-1)
    const F dphi_c = d_axis<F>(Tpm, Tc, Tpp, k, g.np, idp, i2dp);
    const F dth_c = d_axis<F>(Ttm, Tc, Ttp, j, g.nt, idt, i2dt);

    F out = 0, in = 0;
    const F idr = (F)1 / dr;
    // r faces: a = -(T_{i+1} - T_i) / dr, area (r_face)^2 cos theta
    if (hr) {
        F av = -(Trp - Tc) * idr;
        F A = __ldg(a.arf + i) * cth * idr;
        out += A * fmax_(av, (F)0);
        in -= A * fmin(av, (F)0) * P[x + sr];
    }
    if (lr) {
        F av = -(Tc - Trm) * idr;
        F A = __ldg(a.arf + i - 1) * cth * idr;
        out -= A * fmin(av, (F)0);
        in += A * fmax_(av, (F)0) * P[x - sr];
    }
    // theta faces: a = -((1 - 2 xi_h) p_t + 2 eta_h p_p), area r cos theta_face
    if (ht) {
        const long long nn = n + g.np;
        F xh = (F)0.5 * (xic + __ldg(a.xi + nn)), eh = (F)0.5 * (etc + __ldg(a.eta + nn));
        F h3f = h2 * __ldg(a.costf + j);
        F dphi_n = d_axis<F>(Tpm_tp, Ttp, Tpp_tp, k, g.np, idp, i2dp);
        F pt = (Ttp - Tc) * idt / h2;
        F pp = (F)0.5 * (dphi_c + dphi_n) / h3f;
        F av = -(((F)1 - (F)2 * xh) * pt + (F)2 * eh * pp);
        F A = h3f * idt;
        out += A * fmax_(av, (F)0);
        in -= A * fmin(av, (F)0) * P[x + st];
    }
    if (lt) {
        const long long nn = n - g.np;
        F xh = (F)0.5 * (xic + __ldg(a.xi + nn)), eh = (F)0.5 * (etc + __ldg(a.eta + nn));
        F h3f = h2 * __ldg(a.costf + j - 1);
        F dphi_n = d_axis<F>(Tpm_tm, Ttm, Tpp_tm, k, g.np, idp, i2dp);
        F pt = (Tc - Ttm) * idt / h2;
        F pp = (F)0.5 * (dphi_c + dphi_n) / h3f;
        F av = -(((F)1 - (F)2 * xh) * pt + (F)2 * eh * pp);
        F A = h3f * idt;
        out -= A * fmin(av, (F)0);
        in += A * fmax_(av, (F)0) * P[x - st];
    }
    // phi faces: a = -(2 eta_h p_t + (1 + 2 xi_h) p_p), area r
    if (hp) {
        const long long nn = n + 1;
        F xh = (F)0.5 * (xic + __ldg(a.xi + nn)), eh = (F)0.5 * (etc + __ldg(a.eta + nn));
        F dth_n = d_axis<F>(Tpp_tm, Tpp, Tpp_tp, j, g.nt, idt, i2dt);
        F pp = (Tpp - Tc) * idp / h3;
        F pt = (F)0.5 * (dth_c + dth_n) / h2;
        F av = -((F)2 * eh * pt + ((F)1 + (F)2 * xh) * pp);
        F A = h2 * idp;
        out += A * fmax_(av, (F)0);
        in -= A * fmin(av, (F)0) * P[x + sp];
    }
    if (lp) {
        const long long nn = n - 1;
        F xh = (F)0.5 * (xic + __ldg(a.xi + nn)), eh = (F)0.5 * (etc + __ldg(a.eta + nn));
        F dth_n = d_axis<F>(Tpm_tm, Tpm, Tpm_tp, j, g.nt, idt, i2dt);
        F pp = (Tc - Tpm) * idp / h3;
        F pt = (F)0.5 * (dth_c + dth_n) / h2;
        F av = -((F)2 * eh * pt + ((F)1 + (F)2 * xh) * pp);
        F A = h2 * idp;
        out -= A * fmin(av, (F)0);
        in += A * fmax_(av, (F)0) * P[x - sp];
    }
    F js = 0;
    const int h = __ldg(a.sidx + n);
    if (h != kNone) js = a.JS[(long long)h * B + b];
    pold = P[x];
    if (out <= (F)1e-30) return (F)0;
    return (js + in) / out;
}

template <typename F>
__global__ void __launch_bounds__(512) adj_sweep_kernel(AdjArgs<F> a) {
    extern __shared__ unsigned char smem_raw[];
    F *s_err = reinterpret_cast<F *>(smem_raw);
    F *s_pmax = s_err + a.B;
    __shared__ int s_cnt;
    const GridC &g = a.g;
    const int B = a.B;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool lane_ok = tid < (long long)a.slots * B;
    const int b = lane_ok ? (int)(tid % B) : 0;
    const int slot = lane_ok ? (int)(tid / B) : 0;
    const SrcC &sc = a.src[b];
    const int ci = sc.ci, cj = sc.cj, ck = sc.ck;
    barrier_begin();

    for (int it = 0; it < a.max_iter; ++it) {
        const bool active = lane_ok && ((volatile int *)a.conv)[b] == 0;
        F err = 0, pmax = 0;
        for (int o = 0; o < 8; ++o) {
            const bool rr = o & 4, rt = o & 2, rp = o & 1;
            for (int L = 0; L < a.n_planes; ++L) {
                if (active) {
                    const int q1 = __ldg(a.off + L + 1);
                    for (int q = __ldg(a.off + L) + slot; q < q1; q += a.slots) {
                        int aa, bb, cc;
                        unpack(__ldg(a.nodes + q), aa, bb, cc);
                        const int i = rr ? g.nr - 1 - aa : aa;
                        const int j = rt ? g.nt - 1 - bb : bb;
                        const int k = rp ? g.np - 1 - cc : cc;
                        if (in_fixed_set(ci, cj, ck, i, j, k)) continue;
                        const long long n = node_index(g, i, j, k);
                        F pold;
                        F pn = adj_update<F>(a, b, i, j, k, n, pold);
                        a.P[n * B + b] = pn;
                        err = fmax_(err, fabs(pn - pold));
                        if (o == 7) pmax = fmax_(pmax, fabs(pn));
                    }
                }
                if (!grid_barrier(a.bar, a.spin_ns)) return;
            }
        }
        for (int x = threadIdx.x; x < B; x += blockDim.x) { s_err[x] = 0; s_pmax[x] = 0; }
        __syncthreads();
        if (active) {
            atomic_max_nonneg(&s_err[b], err);
            atomic_max_nonneg(&s_pmax[b], pmax);
        }
        __syncthreads();
        for (int x = threadIdx.x; x < B; x += blockDim.x) {
            a.partial[((long long)blockIdx.x * 2) * B + x] = s_err[x];
            a.partial[((long long)blockIdx.x * 2 + 1) * B + x] = s_pmax[x];
        }
        if (!grid_barrier(a.bar, a.spin_ns)) return;
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            for (int x = threadIdx.x; x < B; x += blockDim.x) {
                if (a.conv[x]) continue;
                F m = 0, pm = 0;
                for (int c = 0; c < (int)gridDim.x; ++c) {
                    m = fmax_(m, ((volatile F *)a.partial)[((long long)c * 2) * B + x]);
                    pm = fmax_(pm, ((volatile F *)a.partial)[((long long)c * 2 + 1) * B + x]);
                }
                a.iters[x] = it + 1;
                if (m <= a.tol * pm) a.conv[x] = 1;
                else atomicAdd(&s_cnt, 1);
            }
            __syncthreads();
            if (threadIdx.x == 0) *((volatile int *)a.n_active) = s_cnt;
        }
        if (!grid_barrier(a.bar, a.spin_ns)) return;
        if (*((volatile int *)a.n_active) == 0) break;
    }
    barrier_end(a.bar, gridDim.x);
}

// ------------------------------------------------------------------------ face-coefficient adjoint
//
// The flux velocities of Eq. 5 depend only on T, xi and eta, which stay fixed during the
// adjoint solve. adj_coef_kernel evaluates, once per solve and per (node, source), the
// signed coefficients c_d = A_d a_d / delta_d on the node's +r, +theta and +phi faces (zero
// on the outer boundary) and J_c S_c; the sweep then needs only P and these coefficients:
//   out = sum_d [max(c_d+, 0) - min(c_d-, 0)],
//   in  = sum_d [max(c_d-, 0) P_d- - min(c_d+, 0) P_d+],   P_c = (J_c S_c + in) / out,
// where c_d- is the +face coefficient of the - neighbour (the same face). These are the
// same products as in adj_update, evaluated once instead of every sweep.

template <typename F>
__device__ __forceinline__ void plus_face_coefs(const AdjArgs<F> &a, int b, int i, int j, int k,
                                                long long n, F &cr, F &ct, F &cp) {
    const GridC &g = a.g;
    const long long B = a.B;
    const long long sp = B, st = (long long)g.np * B, sr = (long long)g.nt * g.np * B;
    const long long x = n * B + b;
    const F *T = a.T;
    const bool hr = i < g.nr - 1, ht = j < g.nt - 1, lt = j > 0, hp = k < g.np - 1, lp = k > 0;
    const F dr = (F)g.dr, dt = (F)g.dt, dp = (F)g.dp;
    const F idt = (F)1 / dt, idp = (F)1 / dp, i2dt = (F)0.5 * idt, i2dp = (F)0.5 * idp;
    const F idr = (F)1 / dr;
    const F Tc = T[x];
    const F Ttp = ht ? T[x + st] : Tc, Ttm = lt ? T[x - st] : Tc;
    const F Tpp = hp ? T[x + sp] : Tc, Tpm = lp ? T[x - sp] : Tc;
    const F Tpp_tp = (ht && hp) ? T[x + st + sp] : Tc, Tpm_tp = (ht && lp) ? T[x + st - sp] : Tc;
    const F Tpp_tm = (lt && hp) ? T[x - st + sp] : Tc;
    const F xic = __ldg(a.xi + n), etc = __ldg(a.eta + n);
    const F h2 = __ldg(a.h2 + i), cth = __ldg(a.cost + j);
    const F h3 = h2 * cth;
    const F dphi_c = d_axis<F>(Tpm, Tc, Tpp, k, g.np, idp, i2dp);
    const F dth_c = d_axis<F>(Ttm, Tc, Ttp, j, g.nt, idt, i2dt);
    cr = ct = cp = (F)0;
    if (hr) {
        F av = -(T[x + sr] - Tc) * idr;
        F A = __ldg(a.arf + i) * cth * idr;
        cr = A * av;
    }
    if (ht) {
        const long long nn = n + g.np;
        F xh = (F)0.5 * (xic + __ldg(a.xi + nn)), eh = (F)0.5 * (etc + __ldg(a.eta + nn));
        F h3f = h2 * __ldg(a.costf + j);
        F dphi_n = d_axis<F>(Tpm_tp, Ttp, Tpp_tp, k, g.np, idp, i2dp);
        F pt = (Ttp - Tc) * idt / h2;
        F pp = (F)0.5 * (dphi_c + dphi_n) / h3f;
        F av = -(((F)1 - (F)2 * xh) * pt + (F)2 * eh * pp);
        F A = h3f * idt;
        ct = A * av;
    }
    if (hp) {
        const long long nn = n + 1;
        F xh = (F)0.5 * (xic + __ldg(a.xi + nn)), eh = (F)0.5 * (etc + __ldg(a.eta + nn));
        F dth_n = d_axis<F>(Tpp_tm, Tpp, Tpp_tp, j, g.nt, idt, i2dt);
        F pp = (Tpp - Tc) * idp / h3;
        F pt = (F)0.5 * (dth_c + dth_n) / h2;
        F av = -((F)2 * eh * pt + ((F)1 + (F)2 * xh) * pp);
        F A = h2 * idp;
        cp = A * av;
    }
}


template <typename F> __device__ __forceinline__ F quiet_nan();
template <> __device__ __forceinline__ float quiet_nan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double quiet_nan<double>() {
    return __longlong_as_double(0x7ff8000000000000LL);
}

template <typename F> __global__ void adj_coef_kernel(AdjArgs<F> a) {
    const GridC &g = a.g;
    const long long total = g.N * a.B;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(x % a.B);
        const long long n = x / a.B;
        const int k = (int)(n % g.np);
        const long long t = n / g.np;
        const int j = (int)(t % g.nt), i = (int)(t / g.nt);
        F cr, ct, cp;
        plus_face_coefs<F>(a, b, i, j, k, n, cr, ct, cp);
        const int h = __ldg(a.sidx + n);
        F w = h != kNone ? a.JS[(long long)h * a.B + b] : (F)0;
        const SrcC &sc = a.src[b];
        if (in_fixed_set(sc.ci, sc.cj, sc.ck, i, j, k)) w = quiet_nan<F>();  // never updated
        a.coef[x] = cr;
        a.coef[x + total] = ct;
        a.coef[x + 2 * total] = cp;
        a.coef[x + 3 * total] = w;
    }
}

// Upwind update of one (node, source) from its face coefficients (Eq. 5 discretised as in
// adj_update): c = (+r, +theta, +phi face coefficients, J S), cm = the -r, -theta, -phi
// neighbours' plus-face coefficients, Pn = P at (+r, -r, +theta, -theta, +phi, -phi).
// Rounding-explicit, so both lanes' copies give identical bits.
template <typename F>
__device__ __forceinline__ F face_update(F cx, F cy, F cz, F cw, F cmx, F cmy, F cmz,
                                         const F (&Pn)[6]) {
    const F zero = (F)0;
    const F out = add_(add_(sub_(fmax_(cx, zero), fmin(cmx, zero)),
                            sub_(fmax_(cy, zero), fmin(cmy, zero))),
                       sub_(fmax_(cz, zero), fmin(cmz, zero)));
    const F in = fma_(fmax_(cmx, zero), Pn[1],
                 fma_(-fmin(cx, zero), Pn[0],
                 fma_(fmax_(cmy, zero), Pn[3],
                 fma_(-fmin(cy, zero), Pn[2],
                 fma_(fmax_(cmz, zero), Pn[5], mul_(-fmin(cz, zero), Pn[4]))))));
    return out <= (F)1e-30 ? zero : div_(add_(cw, in), out);
}

// Face-coefficient adjoint sweep. Same organisation as the node-hyperplane forward sweep:
// barrier groups of consecutive sources; a warp covers 64 sources of one node, lane l
// holding sources l and l + 32; on each hyperplane the slots take the nodes slot,
// slot + slots, ...; the schedule is static, so the next node's index and the next
// hyperplane's bounds are read one step ahead. The coefficient planes are separate arrays,
// so every load (a node's four coefficients, each upstream neighbour's one) is a coalesced
// line. Sweeps cover every node (boundary faces carry no flux).
#ifndef TTGB_ADJ_MIN_BLOCKS
#define TTGB_ADJ_MIN_BLOCKS 3
#endif
template <typename F>
__global__ void __launch_bounds__(256, TTGB_ADJ_MIN_BLOCKS) adj_face_kernel(AdjArgs<F> a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_cnt;
    const GridC &g = a.g;
    const int B = a.B;
    const int lgrp = blockIdx.x / a.grp_blocks;         // group within this launch
    const int blk = blockIdx.x - lgrp * a.grp_blocks;
    const int grp = a.grp_base + lgrp;
    const int src0 = grp * a.grp_src;
    const int Bg = min(B, src0 + a.grp_src) - src0;
    if (Bg <= 0) return;
    barrier_begin();
    F *s_err = reinterpret_cast<F *>(smem_raw);
    F *s_pmax = s_err + Bg;
    BarrierState *bar = a.bar + lgrp;  // launches of a chunked solve reuse the same words
    const unsigned nblk = (unsigned)a.grp_blocks;
    const int Bw = ((Bg + 63) >> 6) << 5;               // lanes of one slot
    const int slots = (int)(((long long)a.grp_blocks * blockDim.x) / Bw);
    const long long tid = (long long)blk * blockDim.x + threadIdx.x;
    const bool lane_ok = tid < (long long)slots * Bw;   // uniform over a warp
    const int bl = lane_ok ? (int)(tid % Bw) : 0;
    const int slot = lane_ok ? (int)(tid / Bw) : 0;
    const int lane = threadIdx.x & 31;
    const int l0 = ((bl >> 5) << 6) + lane;
    const bool ok0 = lane_ok && l0 < Bg, ok1 = lane_ok && l0 + 32 < Bg;
    const int b = src0 + (ok0 ? l0 : 0);                // second source: b + 32
    const long long sp = B, st = (long long)g.np * B, sr = (long long)g.nt * g.np * B;
    const long long plane = g.N * B;                    // coefficient plane stride
    const F *cX = a.coef, *cY = a.coef + plane, *cZ = a.coef + 2 * plane, *cW = a.coef + 3 * plane;
    F *P = a.P;

    for (int it = 0; it < a.max_iter; ++it) {
        const bool act0 = ok0 && ((volatile int *)a.conv)[b] == 0;
        const bool act1 = ok1 && ((volatile int *)a.conv)[b + 32] == 0;
        const bool busy = lane_ok && __any_sync(0xffffffffu, act0 || act1);  // uniform
        F err0 = 0, err1 = 0, pmax0 = 0, pmax1 = 0;
        for (int o = 0; o < 8; ++o) {
            const bool rr = o & 4, rt = o & 2, rp = o & 1;
            int qa = __ldg(a.off) + slot, qe = __ldg(a.off + 1);
            unsigned pk = busy && qa < qe ? __ldg(a.nodes + qa) : 0u;
            for (int L = 0; L < a.n_planes; ++L) {
                const bool last = L + 1 == a.n_planes;
                const int qe_next = last ? 0 : __ldg(a.off + L + 2);
                if (busy) {
                    for (int q = qa; q < qe; q += slots) {
                        const int qn = q + slots;
                        const unsigned pkn = qn < qe ? __ldg(a.nodes + qn) : 0u;
                        int aa, bb, cc;
                        unpack(pk, aa, bb, cc);
                        const int i = rr ? g.nr - 1 - aa : aa;
                        const int j = rt ? g.nt - 1 - bb : bb;
                        const int k = rp ? g.np - 1 - cc : cc;
                        const bool hr = i < g.nr - 1, lr = i > 0, ht = j < g.nt - 1, lt = j > 0;
                        const bool hp = k < g.np - 1, lp = k > 0;
                        const long long x = node_index(g, i, j, k) * B + b;
                        // both sources' loads first, then the two updates
                        F cx[2], cy[2], cz[2], w[2], cmx[2], cmy[2], cmz[2], Pn[2][6], po[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (!(h == 0 ? act0 : act1)) continue;
                            const long long y = x + 32 * h;
                            w[h] = cW[y];
                            cx[h] = cX[y];
                            cy[h] = cY[y];
                            cz[h] = cZ[y];
                            cmx[h] = lr ? cX[y - sr] : (F)0;
                            cmy[h] = lt ? cY[y - st] : (F)0;
                            cmz[h] = lp ? cZ[y - sp] : (F)0;
                            Pn[h][0] = hr ? P[y + sr] : (F)0;
                            Pn[h][1] = lr ? P[y - sr] : (F)0;
                            Pn[h][2] = ht ? P[y + st] : (F)0;
                            Pn[h][3] = lt ? P[y - st] : (F)0;
                            Pn[h][4] = hp ? P[y + sp] : (F)0;
                            Pn[h][5] = lp ? P[y - sp] : (F)0;
                            po[h] = P[y];
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (!(h == 0 ? act0 : act1)) continue;
                            if (w[h] != w[h]) continue;  // fixed set: P stays 0
                            const F pn = face_update<F>(cx[h], cy[h], cz[h], w[h], cmx[h],
                                                        cmy[h], cmz[h], Pn[h]);
                            P[x + 32 * h] = pn;
                            if (h == 0) {
                                err0 = fmax_(err0, fabs(pn - po[0]));
                                if (o == 7) pmax0 = fmax_(pmax0, fabs(pn));
                            } else {
                                err1 = fmax_(err1, fabs(pn - po[1]));
                                if (o == 7) pmax1 = fmax_(pmax1, fabs(pn));
                            }
                        }
                        pk = pkn;
                    }
                }
                const int qa_next = qe + slot;
                if (busy && !last && qa_next < qe_next) pk = __ldg(a.nodes + qa_next);
                if (!grid_barrier(bar, a.spin_ns, nblk)) return;
                qa = qa_next;
                qe = qe_next;
            }
        }
        for (int x = threadIdx.x; x < Bg; x += blockDim.x) { s_err[x] = 0; s_pmax[x] = 0; }
        __syncthreads();
        if (act0) {
            atomic_max_nonneg(&s_err[b - src0], err0);
            atomic_max_nonneg(&s_pmax[b - src0], pmax0);
        }
        if (act1) {
            atomic_max_nonneg(&s_err[b + 32 - src0], err1);
            atomic_max_nonneg(&s_pmax[b + 32 - src0], pmax1);
        }
        __syncthreads();
        for (int x = threadIdx.x; x < Bg; x += blockDim.x) {
            a.partial[((long long)blockIdx.x * 2) * B + src0 + x] = s_err[x];
            a.partial[((long long)blockIdx.x * 2 + 1) * B + src0 + x] = s_pmax[x];
        }
        if (!grid_barrier(bar, a.spin_ns, nblk)) return;
        if (blk == 0) {
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            for (int x = src0 + threadIdx.x; x < src0 + Bg; x += blockDim.x) {
                if (a.conv[x]) continue;
                F m = 0, pm = 0;
                for (int c = lgrp * a.grp_blocks; c < (lgrp + 1) * a.grp_blocks; ++c) {
                    m = fmax_(m, ((volatile F *)a.partial)[((long long)c * 2) * B + x]);
                    pm = fmax_(pm, ((volatile F *)a.partial)[((long long)c * 2 + 1) * B + x]);
                }
                a.iters[x] = it + 1;
                if (m <= a.tol * pm) a.conv[x] = 1;
                else atomicAdd(&s_cnt, 1);
            }
            __syncthreads();
            if (threadIdx.x == 0) ((volatile int *)a.n_active)[lgrp] = s_cnt;
        }
        if (!grid_barrier(bar, a.spin_ns, nblk)) return;
        if (((volatile int *)a.n_active)[lgrp] == 0) break;
    }
    barrier_end(bar, nblk);
}

// ------------------------------------------------------------------------ launchers

// The node-hyperplane sweep kernel of one variant.
template <typename F> void *fwd_kernel_ptr(bool refill, bool idx32, int scheme) {
    if (scheme == 3)  // no refill mode
        return idx32 ? (void *)fwd_sweep_kernel<F, unsigned, false, 3>
                     : (void *)fwd_sweep_kernel<F, long long, false, 3>;
    if (scheme == 2)
        return refill ? (idx32 ? (void *)fwd_sweep_kernel<F, unsigned, true, 2>
                               : (void *)fwd_sweep_kernel<F, long long, true, 2>)
                      : (idx32 ? (void *)fwd_sweep_kernel<F, unsigned, false, 2>
                               : (void *)fwd_sweep_kernel<F, long long, false, 2>);
    if (scheme == 1)
        return refill ? (idx32 ? (void *)fwd_sweep_kernel<F, unsigned, true, 1>
                               : (void *)fwd_sweep_kernel<F, long long, true, 1>)
                      : (idx32 ? (void *)fwd_sweep_kernel<F, unsigned, false, 1>
                               : (void *)fwd_sweep_kernel<F, long long, false, 1>);
    return refill ? (idx32 ? (void *)fwd_sweep_kernel<F, unsigned, true, 0>
                           : (void *)fwd_sweep_kernel<F, long long, true, 0>)
                  : (idx32 ? (void *)fwd_sweep_kernel<F, unsigned, false, 0>
                           : (void *)fwd_sweep_kernel<F, long long, false, 0>);
}

template <typename F>
cudaError_t launch_forward(const FwdArgs<F> &a, int grid, int block, cudaStream_t st) {
    void *args[] = {const_cast<FwdArgs<F> *>(&a)};
    const size_t smem = fwd_smem_bytes<F>(a.grp_src, block);
    void *fn = fwd_kernel_ptr<F>(a.refill != 0, a.idx32 != 0, a.scheme);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

template <typename F>
cudaError_t launch_adjoint(const AdjArgs<F> &a, int grid, int block, cudaStream_t st) {
    void *args[] = {const_cast<AdjArgs<F> *>(&a)};
    size_t smem = (size_t)a.B * 2 * sizeof(F);
    return cudaLaunchCooperativeKernel((void *)adj_sweep_kernel<F>, dim3(grid), dim3(block),
                                       args, smem, st);
}

template <typename F> cudaError_t launch_refill_setup(const FwdArgs<F> &a, cudaStream_t st) {
    refill_setup_kernel<F><<<(a.B + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename F> size_t fwd_smem_bytes(int grp_src, int) {
    return fwd_err_bytes<F>(grp_src);
}

template <typename F> int forward_blocks_per_sm(int block, size_t smem, bool idx32, int scheme) {
    int n = 0;
    void *fn = fwd_kernel_ptr<F>(false, idx32, scheme);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem);
    return e == cudaSuccess ? n : 0;
}

template <typename F> int adjoint_blocks_per_sm(int block, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adj_sweep_kernel<F>, block, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

template <typename F, int TA, int TB, int TC> static size_t tiled_smem_bytes(int B) {
    using L = TileSmem<F, TA, TB, TC>;
    return L::err + (size_t)B * sizeof(F) + (size_t)((B + 31) / 32) * sizeof(int);
}

template <typename F> size_t forward_tiled_smem(int shape, int B) {
    switch (shape) {
    case 0: return tiled_smem_bytes<F, 2, 4, 8>(B);
    case 1: return tiled_smem_bytes<F, 4, 4, 4>(B);
    default: return tiled_smem_bytes<F, 2, 8, 8>(B);
    }
}

template <typename F> static const void *tiled_kernel_ptr(int shape) {
    switch (shape) {
    case 0: return (const void *)fwd_tile_kernel<F, 2, 4, 8>;
    case 1: return (const void *)fwd_tile_kernel<F, 4, 4, 4>;
    default: return (const void *)fwd_tile_kernel<F, 2, 8, 8>;
    }
}

template <typename F> int forward_tiled_blocks_per_sm(int shape, int B) {
    const void *k = tiled_kernel_ptr<F>(shape);
    size_t smem = forward_tiled_smem<F>(shape, B);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kTileThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <typename F>
cudaError_t launch_forward_tiled(const CUtensorMap &map_tau, const CUtensorMap &map_rec,
                                 const CUtensorMap &map_t0c, const FwdArgs<F> &a, int shape,
                                 int grid, cudaStream_t st) {
    void *args[] = {const_cast<CUtensorMap *>(&map_tau), const_cast<CUtensorMap *>(&map_rec),
                    const_cast<CUtensorMap *>(&map_t0c), const_cast<FwdArgs<F> *>(&a)};
    return cudaLaunchCooperativeKernel(tiled_kernel_ptr<F>(shape), dim3(grid), dim3(kTileThreads),
                                       args, forward_tiled_smem<F>(shape, a.B), st);
}

template <typename F> cudaError_t launch_t0_cache(const FwdArgs<F> &a, cudaStream_t st) {
    long long total = a.g.N * a.src_n;
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    t0_cache_kernel<F><<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_t0_cache<float>(const FwdArgs<float> &, cudaStream_t);
template cudaError_t launch_t0_cache<double>(const FwdArgs<double> &, cudaStream_t);
template cudaError_t launch_refill_setup<float>(const FwdArgs<float> &, cudaStream_t);
template cudaError_t launch_refill_setup<double>(const FwdArgs<double> &, cudaStream_t);

template <typename F> cudaError_t launch_adjoint_coefs(const AdjArgs<F> &a, cudaStream_t st) {
    long long total = a.g.N * a.B;
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    adj_coef_kernel<F><<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename F>
cudaError_t launch_adjoint_faces(const AdjArgs<F> &a, int grid, int block, cudaStream_t st) {
    void *args[] = {const_cast<AdjArgs<F> *>(&a)};
    size_t smem = (size_t)a.grp_src * 2 * sizeof(F);
    return cudaLaunchCooperativeKernel((void *)adj_face_kernel<F>, dim3(grid), dim3(block), args,
                                       smem, st);
}

template <typename F> int adjoint_faces_blocks_per_sm(int block, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adj_face_kernel<F>, block, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

template size_t forward_tiled_smem<float>(int, int);
template size_t forward_tiled_smem<double>(int, int);
template int forward_tiled_blocks_per_sm<float>(int, int);
template int forward_tiled_blocks_per_sm<double>(int, int);
template cudaError_t launch_forward_tiled<float>(const CUtensorMap &, const CUtensorMap &,
                                                 const CUtensorMap &, const FwdArgs<float> &, int,
                                                 int, cudaStream_t);
template cudaError_t launch_forward_tiled<double>(const CUtensorMap &, const CUtensorMap &,
                                                  const CUtensorMap &, const FwdArgs<double> &,
                                                  int, int, cudaStream_t);
template cudaError_t launch_adjoint_coefs<float>(const AdjArgs<float> &, cudaStream_t);
template cudaError_t launch_adjoint_coefs<double>(const AdjArgs<double> &, cudaStream_t);
template cudaError_t launch_adjoint_faces<float>(const AdjArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_adjoint_faces<double>(const AdjArgs<double> &, int, int, cudaStream_t);
template int adjoint_faces_blocks_per_sm<float>(int, size_t);
template int adjoint_faces_blocks_per_sm<double>(int, size_t);

template cudaError_t launch_forward<float>(const FwdArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_forward<double>(const FwdArgs<double> &, int, int, cudaStream_t);
template cudaError_t launch_adjoint<float>(const AdjArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_adjoint<double>(const AdjArgs<double> &, int, int, cudaStream_t);
template size_t fwd_smem_bytes<float>(int, int);
template size_t fwd_smem_bytes<double>(int, int);
template int forward_blocks_per_sm<float>(int, size_t, bool, int);
template int forward_blocks_per_sm<double>(int, size_t, bool, int);
template int adjoint_blocks_per_sm<float>(int, size_t);
template int adjoint_blocks_per_sm<double>(int, size_t);

}  // namespace ttgb
