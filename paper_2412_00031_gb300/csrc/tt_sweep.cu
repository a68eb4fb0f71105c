// Persistent fast-sweeping kernels of libttgb: the factored Lax-Friedrichs forward sweep
// (Eq. "4", Sec. 3.1) and the upwind adjoint sweep (Eq. 5), both run hyperplane by
// hyperplane (Sec. 3.4) inside one cooperative launch per solve.
//
// Work mapping. Batched fields are stored [node][source]. Thread t of the launch owns one
// source b = t mod B for the whole solve and a slot t / B; on each hyperplane the slots
// stride over the plane's nodes. With B >= 32 a warp reads 32 consecutive sources of one
// node, so every field access is a coalesced 128-byte line and the per-node model values
// are warp-wide broadcasts. Between hyperplanes the launch crosses a bounded grid barrier.
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

__device__ __forceinline__ void unpack(unsigned int pk, int &a, int &b, int &c) {
    a = (int)(pk >> 20);
    b = (int)((pk >> 10) & 1023u);
    c = (int)(pk & 1023u);
}

// ------------------------------------------------------------------------ forward sweep

// Lax-Friedrichs update of tau at interior node (i, j, k) for source b. Dividing the
// update by T0: with u = p0 / T0 and e_d = 1 / (2 delta_d h_d),
//   v = tau_c u + ((tau_d+ - tau_d-) e_d)_d,     H / T0 = sqrt(v^T M v)
//   tau_new = [s / T0 - H / T0 + sum_d c_d (tau_d+ + tau_d-)] / (2 sum_d c_d)
// where c_d = kappa_d e_d and kappa = (1, sqrt(1 - 2 xi), sqrt(1 + 2 xi)) bounds
// |dH/dp_d| / sqrt... (Cauchy-Schwarz), the Lax-Friedrichs viscosity.
template <typename F>
__device__ __forceinline__ F fwd_update(const FwdArgs<F> &a, const SrcReg<F> &S, int b, int i,
                                        int j, int k, long long n, F &told) {
    const long long B = a.B;
    const long long sp = B, st = (long long)a.g.np * B, sr = (long long)a.g.nt * a.g.np * B;
    const long long x = n * B + b;
    F *tau = a.tau;
    F tc = tau[x];
    F trp = tau[x + sr], trm = tau[x - sr];
    F ttp = tau[x + st], ttm = tau[x - st];
    F tpp = tau[x + sp], tpm = tau[x - sp];
    const NodeRec<F> R = a.rec[n];
    F r = __ldg(a.rad + i), cth = __ldg(a.cost + j), sth = __ldg(a.sint + j);
    Vec2<F> tT = a.tabT[(long long)j * B + b];
    Vec2<F> tP = a.tabP[(long long)k * B + b];
    F ur, ut, up;
    F invT0 = factor_T0<F>(S, i, r, cth, sth, tT, tP, a.g.flat != 0, ur, ut, up);
    F vr = tc * ur + (trp - trm) * a.er;
    F vt = tc * ut + (ttp - ttm) * R.et;
    F vp = tc * up + (tpp - tpm) * R.ep;
    F q = vr * vr + ((F)1 - (F)2 * R.xi) * vt * vt + ((F)1 + (F)2 * R.xi) * vp * vp
          + (F)4 * R.eta * vt * vp;
    F H = sqrt_(q);
    F num = R.s * invT0 - H + a.er * (trp + trm) + R.ct * (ttp + ttm) + R.cp * (tpp + tpm);
    told = tc;
    return num * R.invW;
}

// tau on one face layer = max(2 tau_1 - tau_2, tau_2); q enumerates both faces of an axis.
template <typename F>
__device__ __forceinline__ void extrapolate(const FwdArgs<F> &a, const SrcReg<F> &S, int b,
                                            int axis, int slot) {
    const GridC &g = a.g;
    const long long B = a.B;
    int n1, n2, nface;
    long long stride;
    if (axis == 0) { n1 = g.nt; n2 = g.np; nface = g.nr; stride = (long long)g.nt * g.np; }
    else if (axis == 1) { n1 = g.nr; n2 = g.np; nface = g.nt; stride = g.np; }
    else { n1 = g.nr; n2 = g.nt; nface = g.np; stride = 1; }
    const int per_face = n1 * n2;
    for (int q = slot; q < 2 * per_face; q += a.slots) {
        int hi = q >= per_face;
        int rem = hi ? q - per_face : q;
        int u = rem / n2, v = rem - u * n2;
        int f0 = hi ? nface - 1 : 0, f1 = hi ? nface - 2 : 1, f2 = hi ? nface - 3 : 2;
        int i, j, k;
        if (axis == 0) { i = f0; j = u; k = v; }
        else if (axis == 1) { i = u; j = f0; k = v; }
        else { i = u; j = v; k = f0; }
        if (in_fixed_set(S.ci, S.cj, S.ck, i, j, k)) continue;
        long long n = node_index(g, i, j, k);
        long long x0 = n * B + b;
        long long x1 = x0 + (long long)(f1 - f0) * stride * B;
        long long x2 = x0 + (long long)(f2 - f0) * stride * B;
        F t1 = a.tau[x1], t2 = a.tau[x2];
        a.tau[x0] = fmax_((F)2 * t1 - t2, t2);
    }
}

template <typename F>
__global__ void __launch_bounds__(512) fwd_sweep_kernel(FwdArgs<F> a) {
    extern __shared__ unsigned char smem_raw[];
    F *s_err = reinterpret_cast<F *>(smem_raw);
    __shared__ int s_cnt;
    const GridC &g = a.g;
    const int B = a.B;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool lane_ok = tid < (long long)a.slots * B;
    const int b = lane_ok ? (int)(tid % B) : 0;
    const int slot = lane_ok ? (int)(tid / B) : 0;
    const SrcReg<F> S = load_src<F>(a.src, b, g.dr);

    for (int it = 0; it < a.max_iter; ++it) {
        const bool active = lane_ok && ((volatile int *)a.conv)[b] == 0;
        F err = 0;
        for (int o = 0; o < 8; ++o) {
            const bool rr = o & 4, rt = o & 2, rp = o & 1;
            for (int L = 0; L < a.n_planes; ++L) {
                if (active) {
                    const int q1 = __ldg(a.off + L + 1);
                    for (int q = __ldg(a.off + L) + slot; q < q1; q += a.slots) {
                        int aa, bb, cc;
                        unpack(__ldg(a.nodes + q), aa, bb, cc);
                        const int i = rr ? g.nr - 2 - aa : 1 + aa;
                        const int j = rt ? g.nt - 2 - bb : 1 + bb;
                        const int k = rp ? g.np - 2 - cc : 1 + cc;
                        if (in_fixed_set(S.ci, S.cj, S.ck, i, j, k)) continue;
                        const long long n = node_index(g, i, j, k);
                        F told;
                        F tn = fwd_update<F>(a, S, b, i, j, k, n, told);
                        a.tau[n * B + b] = tn;
                        err = fmax_(err, fabs(tn - told));
                    }
                }
                if (!grid_barrier(a.bar, a.spin_ns)) return;
            }
            for (int axis = 0; axis < 3; ++axis) {
                if (active) extrapolate<F>(a, S, b, axis, slot);
                if (!grid_barrier(a.bar, a.spin_ns)) return;
            }
        }
        // Per-source largest update of this iteration: block maximum, then a fixed-order
        // maximum over blocks by block 0, which also decides convergence.
        for (int x = threadIdx.x; x < B; x += blockDim.x) s_err[x] = 0;
        __syncthreads();
        if (active) atomic_max_nonneg(&s_err[b], err);
        __syncthreads();
        for (int x = threadIdx.x; x < B; x += blockDim.x)
            a.partial[(long long)blockIdx.x * B + x] = s_err[x];
        if (!grid_barrier(a.bar, a.spin_ns)) return;
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            for (int x = threadIdx.x; x < B; x += blockDim.x) {
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
}

// ------------------------------------------------------------------------ launchers

template <typename F>
cudaError_t launch_forward(const FwdArgs<F> &a, int grid, int block, cudaStream_t st) {
    void *args[] = {const_cast<FwdArgs<F> *>(&a)};
    size_t smem = (size_t)a.B * sizeof(F);
    return cudaLaunchCooperativeKernel((void *)fwd_sweep_kernel<F>, dim3(grid), dim3(block),
                                       args, smem, st);
}

template <typename F>
cudaError_t launch_adjoint(const AdjArgs<F> &a, int grid, int block, cudaStream_t st) {
    void *args[] = {const_cast<AdjArgs<F> *>(&a)};
    size_t smem = (size_t)a.B * 2 * sizeof(F);
    return cudaLaunchCooperativeKernel((void *)adj_sweep_kernel<F>, dim3(grid), dim3(block),
                                       args, smem, st);
}

template <typename F> int forward_blocks_per_sm(int block, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fwd_sweep_kernel<F>, block, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

template <typename F> int adjoint_blocks_per_sm(int block, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adj_sweep_kernel<F>, block, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

template cudaError_t launch_forward<float>(const FwdArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_forward<double>(const FwdArgs<double> &, int, int, cudaStream_t);
template cudaError_t launch_adjoint<float>(const AdjArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_adjoint<double>(const AdjArgs<double> &, int, int, cudaStream_t);
template int forward_blocks_per_sm<float>(int, size_t);
template int forward_blocks_per_sm<double>(int, size_t);
template int adjoint_blocks_per_sm<float>(int, size_t);
template int adjoint_blocks_per_sm<double>(int, size_t);

}  // namespace ttgb
