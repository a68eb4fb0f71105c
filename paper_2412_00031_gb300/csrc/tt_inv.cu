// The common-receiver differential-time misfit and its adjoint source (Eqs. 4, A4), and the
// regularisation and model update of the inversion step (Sec. 3.3 and step 4 of Sec. 2):
// kernel density (Eq. 19) and the normalisation of the kernels by it (Eq. 18); the
// multiple-grid projection of a kernel onto H offset inversion grids (Eqs. 11-14, 17) and the
// expansion of coefficients back onto the forward grid (Eq. 15); the model update.
//
// Inversion grids: grid h (0 <= h < H) has N nodes per axis at x_a = x_min + (a - h / H) dc,
// dc = (x_max - x_min) / (N - 2), so that every grid covers the forward domain. Along one axis
// the hat function of node a (Eqs. 12-14) is max(0, 1 - |x - x_a| / dc) inside the grid; a
// forward node therefore sees at most two hats per axis and grid. The host tabulates, per
// axis and grid, each forward node's lower coarse node and the two weights; the device
// contracts one axis at a time (projection) or sums the 2 x 2 x 2 products per grid
// (expansion). Every sum runs in a fixed order, so the results do not depend on the launch.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "tt_inv.h"

namespace ttgb {

namespace {

inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Eq. 19 for one batch: Kd[n] += sum over b < B of P[n][b]. One warp per node: lane l adds
// b = l, l + 32, ... in order, then a fixed butterfly.
template <typename F>
__global__ void sum_sources_kernel(long long N, int B, const F *__restrict__ P, double *Kd) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= N) return;
    double acc = 0.0;
    for (int b = lane; b < B; b += 32) acc += (double)P[w * B + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) Kd[w] += acc;
}

// Eqs. 4 and A4. Block b = source b; thread t takes receivers m = t, t + blockDim, ...: for
// the entries of (b, m) (the pairs {b, j} at receiver m, each with dT_obs = T_b^obs - T_j^obs
// and the pair weight w), e = (T_b - T_j) - dT_obs; R[b][m] += gamma sum w e, and the source's
// share of chi_cr is sum w e^2 / 4 (an unordered pair is two ordered terms of weight w / 2,
// split between its two sources). An entry whose other source is out of range sets *bad.
__global__ void misfit_cr_kernel(int n_src, int n_rec, const int *__restrict__ off,
                                 const int *__restrict__ other, const double *__restrict__ dtobs,
                                 const double *__restrict__ w, double gamma,
                                 const double *__restrict__ Tr, double *chi, double *R, int *bad) {
    __shared__ double s[256];
    const int b = blockIdx.x;
    double part = 0.0;
    for (int m = threadIdx.x; m < n_rec; m += blockDim.x) {
        const long long nm = (long long)b * n_rec + m;
        const int q0 = off[nm], q1 = off[nm + 1];
        if (q1 <= q0) continue;
        const double tb = Tr[nm];
        double acc = 0.0;
        for (int q = q0; q < q1; ++q) {
            const int j = other[q];
            if (j < 0 || j >= n_src) {
                atomicExch(bad, 1);
                continue;
            }
            const double e = (tb - Tr[(long long)j * n_rec + m]) - dtobs[q];
            acc += w[q] * e;
            part += 0.25 * w[q] * e * e;
        }
        R[nm] += gamma * acc;
    }
    s[threadIdx.x] = part;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) chi[b] = s[0];
}

// Eq. 18 in place on the three kernels.
__global__ void normalize_kernel(long long N, double *Ks, double *Kxi, double *Keta,
                                 const double *Kd, double eps, double zeta) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double f = 1.0 / pow(Kd[n] + eps, zeta);
    Ks[n] *= f;
    Kxi[n] *= f;
    Keta[n] *= f;
}

// Projection, contraction over phi: T1[h][i][j][c] = sum_k K dV W_p[h][c][k], with
// dV = h2(i)^2 cos(theta_j) dr dtheta dphi.
__global__ void project_phi_kernel(MgDims d, const double *__restrict__ K,
                                   const double *__restrict__ h2, const double *__restrict__ cost,
                                   double dvol, const double *__restrict__ Wp, double *T1) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)d.H * d.nr * d.nt * d.cp;
    if (q >= total) return;
    const int c = (int)(q % d.cp);
    long long r = q / d.cp;
    const int j = (int)(r % d.nt);
    r /= d.nt;
    const int i = (int)(r % d.nr), h = (int)(r / d.nr);
    const double *row = K + ((long long)i * d.nt + j) * d.np;
    const double *w = Wp + ((long long)h * d.cp + c) * d.np;
    double acc = 0.0;
    for (int k = 0; k < d.np; ++k) acc += row[k] * w[k];
    T1[q] = acc * (h2[i] * h2[i] * cost[j] * dvol);
}

// Contraction over theta: T2[h][i][b][c] = sum_j T1[h][i][j][c] W_t[h][b][j].
__global__ void project_theta_kernel(MgDims d, const double *__restrict__ T1,
                                     const double *__restrict__ Wt, double *T2) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)d.H * d.nr * d.ct * d.cp;
    if (q >= total) return;
    const int c = (int)(q % d.cp);
    long long r = q / d.cp;
    const int b = (int)(r % d.ct);
    r /= d.ct;
    const int i = (int)(r % d.nr), h = (int)(r / d.nr);
    const double *src = T1 + (((long long)h * d.nr + i) * d.nt) * d.cp + c;
    const double *w = Wt + ((long long)h * d.ct + b) * d.nt;
    double acc = 0.0;
    for (int j = 0; j < d.nt; ++j) acc += src[(long long)j * d.cp] * w[j];
    T2[q] = acc;
}

// Contraction over r and the 1 / H of Eq. 11: G[h][a][b][c] = sum_i T2[h][i][b][c] W_r[h][a][i] / H.
__global__ void project_r_kernel(MgDims d, const double *__restrict__ T2,
                                 const double *__restrict__ Wr, double *G) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)d.H * d.cr * d.ct * d.cp;
    if (q >= total) return;
    const int c = (int)(q % d.cp);
    long long r = q / d.cp;
    const int b = (int)(r % d.ct);
    r /= d.ct;
    const int a = (int)(r % d.cr), h = (int)(r / d.cr);
    const double *src = T2 + ((long long)h * d.nr * d.ct + b) * d.cp + c;
    const double *w = Wr + ((long long)h * d.cr + a) * d.nr;
    double acc = 0.0;
    for (int i = 0; i < d.nr; ++i) acc += src[(long long)i * d.ct * d.cp] * w[i];
    G[q] = acc / d.H;
}

// Eq. 15: D[i][j][k] = sum over h of the 2 x 2 x 2 products G W_r W_t W_p around the node, / H.
__global__ void expand_kernel(MgDims d, const double *__restrict__ G, const int *__restrict__ lo,
                              const double *__restrict__ Wr, const double *__restrict__ Wt,
                              const double *__restrict__ Wp, double *D) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)d.nr * d.nt * d.np;
    if (n >= N) return;
    const int k = (int)(n % d.np);
    const long long t = n / d.np;
    const int j = (int)(t % d.nt), i = (int)(t / d.nt);
    // lo: [H][nr] then [H][nt] then [H][np], the lower coarse node of each forward node
    const int *lor = lo, *lot = lo + (long long)d.H * d.nr, *lop = lot + (long long)d.H * d.nt;
    double acc = 0.0;
    for (int h = 0; h < d.H; ++h) {
        const int a0 = lor[h * d.nr + i], b0 = lot[h * d.nt + j], c0 = lop[h * d.np + k];
        double sh = 0.0;
        for (int a = a0; a < a0 + 2; ++a) {
            const double wr = Wr[((long long)h * d.cr + a) * d.nr + i];
            for (int b = b0; b < b0 + 2; ++b) {
                const double wt = Wt[((long long)h * d.ct + b) * d.nt + j];
                const double *g = G + (((long long)h * d.cr + a) * d.ct + b) * d.cp;
                sh += wr * wt * (g[c0] * Wp[((long long)h * d.cp + c0) * d.np + k] +
                                 g[c0 + 1] * Wp[((long long)h * d.cp + c0 + 1) * d.np + k]);
            }
        }
        acc += sh;
    }
    D[n] = acc / d.H;
}

// max |x| of each of three FP64 fields: per-block maxima, then one block over them.
__global__ void absmax_partial_kernel(long long N, const double *a, const double *b,
                                      const double *c, double *part) {
    __shared__ double s[3][256];
    double m[3] = {0.0, 0.0, 0.0};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        m[0] = fmax(m[0], fabs(a[n]));
        m[1] = fmax(m[1], fabs(b[n]));
        m[2] = fmax(m[2], fabs(c[n]));
    }
    for (int f = 0; f < 3; ++f) s[f][threadIdx.x] = m[f];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int f = 0; f < 3; ++f) s[f][threadIdx.x] = fmax(s[f][threadIdx.x], s[f][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int f = 0; f < 3; ++f) part[(long long)f * gridDim.x + blockIdx.x] = s[f][0];
}

__global__ void absmax_final_kernel(int nb, const double *part, double *mx) {
    if (threadIdx.x >= 3) return;
    double m = 0.0;
    for (int q = 0; q < nb; ++q) m = fmax(m, part[(long long)threadIdx.x * nb + q]);
    mx[threadIdx.x] = m;
}

// Eq. 18 with eps = eps_rel max(Kd) (Kd >= 0 is a sum of adjoint fields of unit sources): the
// maximum comes from absmax_final_kernel's first slot; 1e-300 when it is 0.
__global__ void normalize_rel_kernel(long long N, double *Ks, double *Kxi, double *Keta,
                                     const double *Kd, const double *mx, double eps_rel,
                                     double zeta) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double e = fmax(eps_rel * mx[0], 1e-300);
    const double f = pow(Kd[n] + e, -zeta);
    Ks[n] *= f;
    Kxi[n] *= f;
    Keta[n] *= f;
}

// Total misfit alpha sum chi[b][0] + beta sum chi[b][1] + gamma sum chi_cr[b] over n sources:
// one block, each thread sums a fixed stride of sources in order, then a fixed tree.
__global__ void misfit_total_kernel(int n, const double *chi, double alpha, double beta,
                                    const double *chi_cr, double gamma, double *out) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        double v = alpha * chi[2 * (long long)b] + beta * chi[2 * (long long)b + 1];
        if (chi_cr) v += gamma * chi_cr[b];
        acc += v;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// The update: s <- s (1 - a D_s / max|D_s|), xi <- xi - a D_xi / max|D_xi|, eta likewise
// (a zero direction leaves its field unchanged).
template <typename F>
__global__ void update_kernel(long long N, F *s, F *xi, F *eta, const double *Ds,
                              const double *Dxi, const double *Deta, const double *mx, double step) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double fs = mx[0] > 0.0 ? step / mx[0] : 0.0;
    const double fx = mx[1] > 0.0 ? step / mx[1] : 0.0;
    const double fe = mx[2] > 0.0 ? step / mx[2] : 0.0;
    s[n] = (F)((double)s[n] * (1.0 - fs * Ds[n]));
    xi[n] = (F)((double)xi[n] - fx * Dxi[n]);
    eta[n] = (F)((double)eta[n] - fe * Deta[n]);
}

}  // namespace

// Per-axis tables of the H grids of `c` nodes over `n` forward nodes: W[h][a][i] (the hat
// of coarse node a at forward node i, in the axis coordinate scaled to [0, 1]) and lo[h][i]
// (the coarse node below forward node i: its hats are lo and lo + 1).
void mgrid_axis_tables(int n, int c, int H, std::vector<double> &W, std::vector<int> &lo) {
    W.assign((size_t)H * c * n, 0.0);
    lo.assign((size_t)H * n, 0);
    const double dc = 1.0 / (c - 2);
    for (int h = 0; h < H; ++h)
        for (int i = 0; i < n; ++i) {
            const double x = (double)i / (n - 1);
            const double u = x / dc + (double)h / H;       // position in coarse cells from node 0
            int a = (int)std::floor(u);
            if (a > c - 2) a = c - 2;
            if (a < 0) a = 0;
            lo[(size_t)h * n + i] = a;
            for (int q = a; q <= a + 1; ++q) {
                const double xa = (q - (double)h / H) * dc;
                const double v = 1.0 - std::fabs(x - xa) / dc;
                W[((size_t)h * c + q) * n + i] = v > 0.0 ? v : 0.0;
            }
        }
}

cudaError_t run_misfit_cr(int n_src, int n_rec, const int *off, const int *other,
                          const double *dtobs, const double *w, double gamma, const double *Tr,
                          double *chi, double *R, int *bad, cudaStream_t st) {
    misfit_cr_kernel<<<n_src, 256, 0, st>>>(n_src, n_rec, off, other, dtobs, w, gamma, Tr, chi, R, bad);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_kernel_density(long long N, int B, const F *P, double *Kd, cudaStream_t st) {
    sum_sources_kernel<F><<<nblocks(N * 32, 256), 256, 0, st>>>(N, B, P, Kd);
    return cudaGetLastError();
}

cudaError_t run_kernel_normalize(long long N, double *Ks, double *Kxi, double *Keta,
                                 const double *Kd, double eps, double zeta, cudaStream_t st) {
    normalize_kernel<<<nblocks(N, 256), 256, 0, st>>>(N, Ks, Kxi, Keta, Kd, eps, zeta);
    return cudaGetLastError();
}

cudaError_t run_mgrid_project(const MgDims &d, const double *K, const double *h2,
                              const double *cost, double dvol, const double *Wr,
                              const double *Wt, const double *Wp, double *T1, double *T2,
                              double *G, cudaStream_t st) {
    const long long n1 = (long long)d.H * d.nr * d.nt * d.cp;
    const long long n2 = (long long)d.H * d.nr * d.ct * d.cp;
    const long long n3 = (long long)d.H * d.cr * d.ct * d.cp;
    project_phi_kernel<<<nblocks(n1, 256), 256, 0, st>>>(d, K, h2, cost, dvol, Wp, T1);
    project_theta_kernel<<<nblocks(n2, 256), 256, 0, st>>>(d, T1, Wt, T2);
    project_r_kernel<<<nblocks(n3, 256), 256, 0, st>>>(d, T2, Wr, G);
    return cudaGetLastError();
}

cudaError_t run_mgrid_expand(const MgDims &d, const double *G, const int *lo, const double *Wr,
                             const double *Wt, const double *Wp, double *D, cudaStream_t st) {
    expand_kernel<<<nblocks((long long)d.nr * d.nt * d.np, 256), 256, 0, st>>>(d, G, lo, Wr, Wt, Wp, D);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_model_update(long long N, F *s, F *xi, F *eta, const double *Ds,
                             const double *Dxi, const double *Deta, double step, double *part,
                             int n_part, cudaStream_t st) {
    absmax_partial_kernel<<<n_part, 256, 0, st>>>(N, Ds, Dxi, Deta, part);
    absmax_final_kernel<<<1, 32, 0, st>>>(n_part, part, part + 3 * n_part);
    update_kernel<F><<<nblocks(N, 256), 256, 0, st>>>(N, s, xi, eta, Ds, Dxi, Deta,
                                                      part + 3 * n_part, step);
    return cudaGetLastError();
}

cudaError_t run_kernel_normalize_rel(long long N, double *Ks, double *Kxi, double *Keta,
                                     const double *Kd, double eps_rel, double zeta, double *part,
                                     int n_part, cudaStream_t st) {
    // the partial maxima of Kd (the kernel takes three fields: Kd three times)
    absmax_partial_kernel<<<n_part, 256, 0, st>>>(N, Kd, Kd, Kd, part);
    absmax_final_kernel<<<1, 32, 0, st>>>(n_part, part, part + 3 * n_part);
    normalize_rel_kernel<<<nblocks(N, 256), 256, 0, st>>>(N, Ks, Kxi, Keta, Kd,
                                                          part + 3 * n_part, eps_rel, zeta);
    return cudaGetLastError();
}

cudaError_t run_misfit_total(int n, const double *chi, double alpha, double beta,
                             const double *chi_cr, double gamma, double *out, cudaStream_t st) {
    misfit_total_kernel<<<1, 256, 0, st>>>(n, chi, alpha, beta, chi_cr, gamma, out);
    return cudaGetLastError();
}

template cudaError_t run_kernel_density<float>(long long, int, const float *, double *, cudaStream_t);
template cudaError_t run_kernel_density<double>(long long, int, const double *, double *, cudaStream_t);
template cudaError_t run_model_update<float>(long long, float *, float *, float *, const double *,
                                             const double *, const double *, double, double *,
                                             int, cudaStream_t);
template cudaError_t run_model_update<double>(long long, double *, double *, double *,
                                              const double *, const double *, const double *,
                                              double, double *, int, cudaStream_t);

}  // namespace ttgb
