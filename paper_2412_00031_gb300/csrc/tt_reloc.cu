// Earthquake location and origin-time kernels (Eq. 10, Appendix B, Eqs. B1-B11).
//
// By reciprocity the time from event n to receiver m is Gamma_m(x_n), the traveltime of a
// wavefront started at receiver m, so the arrivals are Gamma_m(x_n) + tau_n (origin time).
// With R_{n,m} = dchi / dT_n(x_m), the adjoint sources of Eqs. A2-A4 evaluated on those
// arrivals:
//   K_x,n   = sum_m R_{n,m} grad Gamma_m(x_n)    (Eqs. B5-B7)
//   K_tau,n = sum_m R_{n,m}                      (Eqs. B9-B11)
// Gamma_m(x) is the trilinear interpolant of the nodal field (index space, as for receiver
// times) and grad Gamma_m its gradient in physical components (d/dr, d/(r dtheta),
// d/(r cos(theta) dphi)) at the point. K_x is then the derivative of the discrete misfit
// with respect to the event position.
#include <cuda_runtime.h>

#include "tt_reloc.h"

namespace ttgb {

namespace {

constexpr double kDeg = 3.14159265358979323846 / 180.0;

// Fractional index of (depth, lat, lon), the cell (lower corner clamped to the grid) and the
// position u within it; *out = true when the point lies outside the grid (by more than
// 1e-9 of a cell). Each operation is rounded on its own (no fused multiply-add), so the
// index, and with it the choice of cell at a cell face where the gradient jumps, is the
// one that the same expression gives in plain IEEE double arithmetic.
__device__ inline void point_cell(const GridC &g, const double *p, int base[3], double u[3],
                                  bool &out) {
    const double f[3] = {__ddiv_rn(__dsub_rn(__dsub_rn(g.re, p[0]), g.r0), g.dr),
                         __ddiv_rn(__dsub_rn(__dmul_rn(p[1], kDeg), g.t0), g.dt),
                         __ddiv_rn(__dsub_rn(__dmul_rn(p[2], kDeg), g.p0), g.dp)};
    const int n[3] = {g.nr, g.nt, g.np};
    const double eps = 1e-9;
    out = false;
    for (int a = 0; a < 3; ++a) {
        if (!(f[a] >= -eps && f[a] <= n[a] - 1 + eps)) out = true;
        double fl = floor(f[a]);
        int i0 = fl != fl ? 0 : (fl < 0.0 ? 0 : (fl > n[a] - 2 ? n[a] - 2 : (int)fl));
        base[a] = i0;
        u[a] = out ? 0.0 : f[a] - i0;
    }
}

// One warp per point; lanes stride over the fields (consecutive fields of a node are
// consecutive in memory).
template <typename F>
__global__ void field_at_points_kernel(GridC g, int M, int n_pts, const F *G, const double *pts,
                                       double *val, double *grad, int *bad) {
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= n_pts) return;
    int base[3];
    double u[3];
    bool out;
    point_cell(g, pts + 3 * q, base, u, out);
    if (out && lane == 0) atomicExch(bad, 1);
    const double r = g.re - pts[3 * q];
    const double th = pts[3 * q + 1] * kDeg;
    const double h2 = g.flat ? g.re : r;
    const double h3 = g.flat ? g.re : r * cos(th);
    const double sr = 1.0 / g.dr, st = 1.0 / (g.dt * h2), sp = 1.0 / (g.dp * h3);
    long long node[8];
    for (int c = 0; c < 8; ++c)
        node[c] = node_index(g, base[0] + ((c >> 2) & 1), base[1] + ((c >> 1) & 1),
                             base[2] + (c & 1));
    for (int m = lane; m < M; m += 32) {
        double v = 0.0, di = 0.0, dj = 0.0, dk = 0.0;
        for (int c = 0; c < 8; ++c) {
            const double f = (double)G[node[c] * M + m];
            const double wr = (c & 4) ? u[0] : 1.0 - u[0], ar = (c & 4) ? 1.0 : -1.0;
            const double wt = (c & 2) ? u[1] : 1.0 - u[1], at = (c & 2) ? 1.0 : -1.0;
            const double wp = (c & 1) ? u[2] : 1.0 - u[2], ap = (c & 1) ? 1.0 : -1.0;
            v += wr * wt * wp * f;
            di += ar * wt * wp * f;
            dj += wr * at * wp * f;
            dk += wr * wt * ap * f;
        }
        const long long o = (long long)q * M + m;
        val[o] = v;
        grad[3 * o] = di * sr;
        grad[3 * o + 1] = dj * st;
        grad[3 * o + 2] = dk * sp;
    }
}

// One warp per event; lanes stride over the receivers and the four sums close with a
// fixed shuffle tree, so the result is bitwise reproducible.
__global__ void reloc_kernels_kernel(int n_src, int n_rec, const double *R, const double *grad,
                                     double *Kx, double *Kt) {
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (n >= n_src) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, at = 0.0;
    for (int m = lane; m < n_rec; m += 32) {
        const long long o = (long long)n * n_rec + m;
        const double rr = R[o];
        a0 += rr * grad[3 * o];
        a1 += rr * grad[3 * o + 1];
        a2 += rr * grad[3 * o + 2];
        at += rr;
    }
    for (int s = 16; s > 0; s >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, s);
        a1 += __shfl_xor_sync(0xffffffffu, a1, s);
        a2 += __shfl_xor_sync(0xffffffffu, a2, s);
        at += __shfl_xor_sync(0xffffffffu, at, s);
    }
    if (lane == 0) {
        Kx[3 * n] = a0;
        Kx[3 * n + 1] = a1;
        Kx[3 * n + 2] = a2;
        Kt[n] = at;
    }
}

constexpr int kUpdThreads = 256;

// One block: the largest |K_x,n| and |K_tau,n| (a fixed-order tree), then every event moves
// by -step_km K_x,n / max (km, physical components), clamped to the grid, and its origin time
// by -step_s K_tau,n / max.
__global__ void __launch_bounds__(kUpdThreads)
reloc_update_kernel(GridC g, GridBox box, int n_src, double *pts, double *otime,
                    const double *Kx, const double *Kt, double step_km, double step_s) {
    __shared__ double sx[kUpdThreads], stt[kUpdThreads];
    double mx = 0.0, mt = 0.0;
    for (int n = threadIdx.x; n < n_src; n += kUpdThreads) {
        const double k0 = Kx[3 * n], k1 = Kx[3 * n + 1], k2 = Kx[3 * n + 2];
        mx = fmax(mx, sqrt(k0 * k0 + k1 * k1 + k2 * k2));
        mt = fmax(mt, fabs(Kt[n]));
    }
    sx[threadIdx.x] = mx;
    stt[threadIdx.x] = mt;
    __syncthreads();
    for (int s = kUpdThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sx[threadIdx.x] = fmax(sx[threadIdx.x], sx[threadIdx.x + s]);
            stt[threadIdx.x] = fmax(stt[threadIdx.x], stt[threadIdx.x + s]);
        }
        __syncthreads();
    }
    mx = sx[0];
    mt = stt[0];
    for (int n = threadIdx.x; n < n_src; n += kUpdThreads) {
        double *p = pts + 3 * n;
        if (mx > 0.0) {
            const double d0 = -step_km * Kx[3 * n] / mx;
            const double d1 = -step_km * Kx[3 * n + 1] / mx;
            const double d2 = -step_km * Kx[3 * n + 2] / mx;
            const double r = g.re - p[0];
            const double th = p[1] * kDeg;
            const double h2 = g.flat ? g.re : r;
            const double h3 = g.flat ? g.re : r * cos(th);
            const double dep = p[0] - d0;  // depth = R_E - r: a step up lowers it
            const double lat = p[1] + d1 / h2 / kDeg;
            const double lon = p[2] + d2 / h3 / kDeg;
            p[0] = fmin(fmax(dep, box.lo[0]), box.hi[0]);
            p[1] = fmin(fmax(lat, box.lo[1]), box.hi[1]);
            p[2] = fmin(fmax(lon, box.lo[2]), box.hi[2]);
        }
        if (mt > 0.0 && otime) otime[n] -= step_s * Kt[n] / mt;
    }
}

}  // namespace

template <typename F>
cudaError_t run_field_at_points(const GridC &g, int M, int n_pts, const void *G,
                                const double *pts, double *val, double *grad, int *bad,
                                cudaStream_t st) {
    const int warps = 8;
    const unsigned blocks = (unsigned)((n_pts + warps - 1) / warps);
    field_at_points_kernel<F><<<blocks, warps * 32, 0, st>>>(g, M, n_pts, (const F *)G, pts, val,
                                                             grad, bad);
    return cudaGetLastError();
}

cudaError_t run_reloc_kernels(int n_src, int n_rec, const double *R, const double *grad,
                              double *Kx, double *Kt, cudaStream_t st) {
    const int warps = 8;
    const unsigned blocks = (unsigned)((n_src + warps - 1) / warps);
    reloc_kernels_kernel<<<blocks, warps * 32, 0, st>>>(n_src, n_rec, R, grad, Kx, Kt);
    return cudaGetLastError();
}

cudaError_t run_reloc_update(const GridC &g, const GridBox &box, int n_src, double *pts,
                             double *otime, const double *Kx, const double *Kt, double step_km,
                             double step_s, cudaStream_t st) {
    reloc_update_kernel<<<1, kUpdThreads, 0, st>>>(g, box, n_src, pts, otime, Kx, Kt, step_km,
                                                   step_s);
    return cudaGetLastError();
}

template cudaError_t run_field_at_points<float>(const GridC &, int, int, const void *,
                                                const double *, double *, double *, int *,
                                                cudaStream_t);
template cudaError_t run_field_at_points<double>(const GridC &, int, int, const void *,
                                                 const double *, double *, double *, int *,
                                                 cudaStream_t);

}  // namespace ttgb
