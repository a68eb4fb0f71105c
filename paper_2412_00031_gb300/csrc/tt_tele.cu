// Teleseismic events: the 2-D traveltimes of an event outside the region in a 1-D model
// s(r), in (r, Delta) with Delta the epicentral angle, and their interpolation onto the
// region's nodes (the Dirichlet data of the region's faces and the interior's start).
//
// The 2-D solve is factored (T = T0 tau, T0 = s(r_s) x chord from the event) with the
// Godunov update in two dimensions: one-sided differences toward the upwind neighbour of
// each axis (the one with the smaller first-order estimate of T), the smallest causal root
// over the axis subsets, solved for the increment tau - tau_c. The axis Delta = 0 is a
// mirror; the faces r = r_min, r = r_max and Delta = Delta_max take tau_0 = max(2 tau_1 -
// tau_2, tau_2) after each sweep; the 3 x 2 nodes next to the event keep tau = 1. The four
// orderings sweep the anti-diagonals of the (r, Delta) grid, which gives the lexicographic
// order's result for this five-point stencil. One block per event: its sweeps need only
// block barriers, and every loop is bounded by max_iter.
#include <cuda_runtime.h>

#include "tt_common.cuh"
#include "tt_tele.h"

namespace ttgb {

namespace {

constexpr int kTeleThreads = 512;

template <typename F>
__device__ __forceinline__ F s_of_r(int n_r, F r_min, F dr, const F *s_r, F r) {
    const F f = div_(sub_(r, r_min), dr);
    int i = (int)floor(f);
    i = i < 0 ? 0 : (i > n_r - 2 ? n_r - 2 : i);
    const F w = sub_(f, (F)i);
    return fma_(w, s_r[i + 1], mul_(sub_((F)1, w), s_r[i]));
}

template <typename F> __device__ __forceinline__ F sin_(F x);
template <> __device__ __forceinline__ float sin_(float x) { return sinf(x); }
template <> __device__ __forceinline__ double sin_(double x) { return sin(x); }

// The chord from the event (r_s, 0) to (r, D), squared, and u = grad T0 / T0 in physical
// components (d/dr, d/(r dD)), written without cancellation near the event:
// L^2 = (r - r_s)^2 + 4 r r_s sin^2(D/2), r - r_s cos D = (r - r_s) + 2 r_s sin^2(D/2).
template <typename F>
__device__ __forceinline__ void chord(F r, F r_s, F D, F &L2, F &ur, F &ud) {
    const F h = sin_(mul_((F)0.5, D));
    const F h2 = mul_(h, h);
    const F dr = sub_(r, r_s);
    L2 = fma_(dr, dr, mul_(mul_((F)4 * r, r_s), h2));
    const F inv = div_((F)1, L2);
    ur = mul_(fma_((F)2 * r_s, h2, dr), inv);
    ud = mul_(mul_(r_s, sin_(D)), inv);
}

template <typename F>
__device__ F god2d(F r, F D, F r_s, F s_s, F s_here, F dr, F dd, F tc, F lo0, F hi0, F lo1,
                   F hi1) {
    F L2, u0, u1;
    chord<F>(r, r_s, D, L2, u0, u1);
    const F u[2] = {u0, u1};
    const F e[2] = {div_((F)1, dr), div_((F)1, mul_(r, dd))};
    const F lo[2] = {lo0, lo1}, hi[2] = {hi0, hi1};
    F a[2], c[2], sg[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const bool lower = mul_(lo[d], sub_(e[d], u[d])) <= mul_(hi[d], add_(e[d], u[d]));
        sg[d] = lower ? (F)1 : (F)-1;
        const F se = mul_(sg[d], e[d]);
        a[d] = add_(se, u[d]);
        c[d] = fma_(u[d], tc, mul_(se, sub_(tc, lower ? lo[d] : hi[d])));
    }
    const F rhs = div_(s_here, mul_(s_s, sqrt_(L2)));
    const F r2 = mul_(rhs, rhs);
    F bestN = (F)0, bestD = (F)1;
    bool found = false;
    // both axes first: a causal root there is the smallest (each single axis's form never
    // exceeds the full one)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int mask = q == 0 ? 3 : q;            // {r, D}, then {r}, {D}
        if (q == 1 && found) break;                  // a causal root on both axes
        F A = 0, B = 0, C = -r2;
#pragma unroll
        for (int d = 0; d < 2; ++d)
            if (mask >> d & 1) {
                A = fma_(a[d], a[d], A);
                B = fma_(a[d], c[d], B);
                C = fma_(c[d], c[d], C);
            }
        const F disc = fma_(B, B, -mul_(A, C));
        if (!(A > (F)0) || disc < (F)0) continue;
        const F qd = sqrt_(disc);
        const bool pos = B >= (F)0;
        const F N = pos ? -C : sub_(qd, B);
        const F Dn = pos ? add_(B, qd) : A;
        if (!(Dn > (F)0)) continue;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 2; ++d)
            if ((mask >> d & 1) && mul_(sg[d], fma_(a[d], N, mul_(c[d], Dn))) < (F)0) ok = false;
        if (ok && (!found || mul_(N, bestD) < mul_(bestN, Dn))) {
            bestN = N;
            bestD = Dn;
            found = true;
        }
    }
    return found ? add_(tc, div_(bestN, bestD)) : tc;
}

template <typename F>
__global__ void __launch_bounds__(kTeleThreads)
tele2d_kernel(int n_r, int n_d, F r_min, F dr, F dd, const F *s_r, const double *r_src,
              F tol, int max_iter, F *tau_all, F *T_all, int *iters) {
    __shared__ F red[kTeleThreads];
    __shared__ int done;
    const int ev = blockIdx.x;
    const int tid = threadIdx.x;
    const long long NN = (long long)n_r * n_d;
    F *tau = tau_all + ev * NN;
    const F r_s = (F)r_src[ev];
    const F s_s = s_of_r<F>(n_r, r_min, dr, s_r, r_s);
    int is = (int)floor((double)((r_s - r_min) / dr) + 0.5);
    is = is < 0 ? 0 : (is > n_r - 1 ? n_r - 1 : is);
    for (long long q = tid; q < NN; q += kTeleThreads) tau[q] = (F)1;
    if (tid == 0) done = 0;
    __syncthreads();
    int it = 0;
    for (; it < max_iter; ++it) {
        F err = (F)0;
        for (int o = 0; o < 4; ++o) {
            const bool up_i = !(o & 2), up_j = !(o & 1);
            const int na = n_r - 2, nb = n_d - 1;       // interior rows, swept columns
            for (int L = 0; L <= na + nb - 2; ++L) {
                const int a0 = L - (nb - 1) > 0 ? L - (nb - 1) : 0;
                const int a1 = L < na - 1 ? L : na - 1;
                for (int a = a0 + tid; a <= a1; a += kTeleThreads) {
                    const int b = L - a;
                    const int i = up_i ? 1 + a : n_r - 2 - a;
                    const int j = up_j ? b : n_d - 2 - b;
                    if (abs(i - is) <= 1 && j <= 1) continue;
                    const long long c = (long long)i * n_d + j;
                    const F r = fma_((F)i, dr, r_min), D = mul_((F)j, dd);
                    const F tc = tau[c];
                    const F v = god2d<F>(r, D, r_s, s_s, s_of_r<F>(n_r, r_min, dr, s_r, r), dr,
                                         dd, tc, tau[c - n_d], tau[c + n_d],
                                         tau[(long long)i * n_d + (j > 0 ? j - 1 : 1)], tau[c + 1]);
                    err = fmax(err, fabs(v - tc));
                    tau[c] = v;
                }
                __syncthreads();
            }
            // faces r = r_min and r = r_max (all Delta), then Delta = Delta_max (all r)
            for (int j = tid; j < n_d; j += kTeleThreads) {
                if (!(abs(0 - is) <= 1 && j <= 1))
                    tau[j] = fmax(2 * tau[n_d + j] - tau[2 * n_d + j], tau[2 * n_d + j]);
                if (!(abs(n_r - 1 - is) <= 1 && j <= 1)) {
                    const long long t1 = (long long)(n_r - 2) * n_d + j, t2 = (long long)(n_r - 3) * n_d + j;
                    tau[(long long)(n_r - 1) * n_d + j] = fmax(2 * tau[t1] - tau[t2], tau[t2]);
                }
            }
            __syncthreads();
            for (int i = tid; i < n_r; i += kTeleThreads) {
                const long long row = (long long)i * n_d;
                tau[row + n_d - 1] = fmax(2 * tau[row + n_d - 2] - tau[row + n_d - 3], tau[row + n_d - 3]);
            }
            __syncthreads();
        }
        // block maximum of the iteration's changes (fixed order)
        red[tid] = err;
        __syncthreads();
        for (int s = kTeleThreads / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
            __syncthreads();
        }
        if (tid == 0) done = red[0] < tol;
        __syncthreads();
        if (done) {
            ++it;
            break;
        }
        __syncthreads();
    }
    if (tid == 0) iters[ev] = it;
    for (long long q = tid; q < NN; q += kTeleThreads) {
        const int i = (int)(q / n_d), j = (int)(q % n_d);
        F L2, u0, u1;
        chord<F>(fma_((F)i, dr, r_min), r_s, mul_((F)j, dd), L2, u0, u1);
        T_all[ev * NN + q] = mul_(mul_(s_s, sqrt_(L2)), tau[q]);
    }
}

// The region's nodes (batched [node][event]): bilinear interpolation of each event's 2-D
// times at the node's radius and epicentral angle.
template <typename F>
__global__ void region_times_kernel(GridC g, int n_r, int n_d, double r_min, double dr2,
                                    double dd, const F *T2, int n_ev, const double *ev_ll,
                                    F *T) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= g.N * n_ev) return;
    const long long n = q / n_ev;
    const int e = (int)(q % n_ev);
    const int k = (int)(n % g.np);
    const long long t = n / g.np;
    const int j = (int)(t % g.nt), i = (int)(t / g.nt);
    const double r = g.r0 + i * g.dr, th = g.t0 + j * g.dt, ph = g.p0 + k * g.dp;
    const double ts = ev_ll[2 * e], ps = ev_ll[2 * e + 1];
    double cd = sin(th) * sin(ts) + cos(th) * cos(ts) * cos(ph - ps);
    cd = cd > 1.0 ? 1.0 : (cd < -1.0 ? -1.0 : cd);
    const double D = acos(cd);
    const double fr = (r - r_min) / dr2, fd = D / dd;
    int a = (int)floor(fr), b = (int)floor(fd);
    a = a < 0 ? 0 : (a > n_r - 2 ? n_r - 2 : a);
    b = b < 0 ? 0 : (b > n_d - 2 ? n_d - 2 : b);
    const double u = fr - a, v = fd - b;
    const F *Te = T2 + (long long)e * n_r * n_d;
    const long long c = (long long)a * n_d + b;
    T[q] = (F)((1 - u) * (1 - v) * (double)Te[c] + u * (1 - v) * (double)Te[c + n_d] +
               (1 - u) * v * (double)Te[c + 1] + u * v * (double)Te[c + n_d + 1]);
}

// The region's solve of an event only sees differences of T (the Lax-Friedrichs update is
// unchanged when a constant is added to T), so it runs on T - c_e with c_e = T at node 0 (a
// corner: face data, held fixed). Teleseismic times of a few hundred seconds then become
// values within the region's spread of times, whose FP32 resolution is several times finer.
template <typename F>
__global__ void tele_shift_save_kernel(int n_ev, const F *T, F *c) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_ev) c[e] = T[e];
}
template <typename F>
__global__ void tele_shift_kernel(long long N, int n_ev, F *T, const F *c, int sign) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N * n_ev) return;
    const int e = (int)(q % n_ev);
    T[q] = sign < 0 ? T[q] - c[e] : T[q] + c[e];
}

}  // namespace

template <typename F>
cudaError_t run_tele_shift(long long N, int n_ev, void *T, void *c, int sign, cudaStream_t st) {
    if (sign < 0) tele_shift_save_kernel<F><<<(n_ev + 255) / 256, 256, 0, st>>>(n_ev, (const F *)T, (F *)c);
    const long long total = N * n_ev;
    tele_shift_kernel<F><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(N, n_ev, (F *)T, (const F *)c,
                                                                         sign);
    return cudaGetLastError();
}
template cudaError_t run_tele_shift<float>(long long, int, void *, void *, int, cudaStream_t);
template cudaError_t run_tele_shift<double>(long long, int, void *, void *, int, cudaStream_t);

template <typename F>
cudaError_t run_tele2d(int n_r, int n_d, double r_min, double dr, double dd, const void *s_r,
                       const double *r_src, int n_ev, double tol, int max_iter, void *tau,
                       void *T, int *iters, cudaStream_t st) {
    tele2d_kernel<F><<<n_ev, kTeleThreads, 0, st>>>(n_r, n_d, (F)r_min, (F)dr, (F)dd,
                                                    (const F *)s_r, r_src, (F)tol, max_iter,
                                                    (F *)tau, (F *)T, iters);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_region_times(const GridC &g, int n_r, int n_d, double r_min, double dr2,
                             double dd, const void *T2, int n_ev, const double *ev_ll, void *T,
                             cudaStream_t st) {
    const long long total = g.N * n_ev;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    region_times_kernel<F><<<blocks, 256, 0, st>>>(g, n_r, n_d, r_min, dr2, dd, (const F *)T2,
                                                   n_ev, ev_ll, (F *)T);
    return cudaGetLastError();
}

template cudaError_t run_tele2d<float>(int, int, double, double, double, const void *,
                                       const double *, int, double, int, void *, void *, int *,
                                       cudaStream_t);
template cudaError_t run_tele2d<double>(int, int, double, double, double, const void *,
                                        const double *, int, double, int, void *, void *, int *,
                                        cudaStream_t);
template cudaError_t run_region_times<float>(const GridC &, int, int, double, double, double,
                                             const void *, int, const double *, void *,
                                             cudaStream_t);
template cudaError_t run_region_times<double>(const GridC &, int, int, double, double, double,
                                              const void *, int, const double *, void *,
                                              cudaStream_t);

}  // namespace ttgb
