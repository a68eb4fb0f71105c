// Warm-start network kernels of libttgb. The network predicts the factored correction tau
// of Sec. 3.1 (T = T0 tau) from six local channels per node (s / s0 - 1, xi, eta and the
// offset to the source in the source's frame); four 3x3x3 convolutions 6 -> 32 -> 32 -> 32
// -> 1 with ReLU between them, zero padding outside the grid. Training (MSE on tau - 1)
// runs here too: the convolution, its input gradient (a convolution with flipped,
// transposed weights), its weight gradient (a deterministic two-stage reduction over all
// positions) and Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tt_net.h"

namespace ttgb {

namespace {

// Output tile of one convolution block: 4 x 4 x 8 nodes (z = r, y = theta, x = phi), one
// node per thread; its input with a one-node halo is 6 x 6 x 10 nodes.
constexpr int kTZ = 4, kTY = 4, kTX = 8;
constexpr int kHZ = kTZ + 2, kHY = kTY + 2, kHX = kTX + 2;
constexpr int kHalo = kHZ * kHY * kHX;
constexpr int kCK = 8;  // input channels staged per pass
constexpr int kConvThreads = kTZ * kTY * kTX;

// FP32 3x3x3 convolution of the training path (the inference path runs on the tensor cores,
// tt_umma.cu).
template <int COUT>
__global__ void __launch_bounds__(kConvThreads)
    conv3d_kernel(ConvDims d, int cin, const float *__restrict__ in, int relu_in,
                  const float *__restrict__ w, const float *__restrict__ bias,
                  const float *__restrict__ gate, float *__restrict__ out) {
    __shared__ float s_in[kHalo * (kCK + 1)];  // odd channel stride: no bank conflicts
    __shared__ __align__(16) float s_w[27 * kCK * COUT];
    const int tiles_x = (d.W + kTX - 1) / kTX, tiles_y = (d.H + kTY - 1) / kTY;
    int tile = blockIdx.x;
    const int x0 = (tile % tiles_x) * kTX;
    tile /= tiles_x;
    const int y0 = (tile % tiles_y) * kTY;
    const int z0 = (tile / tiles_y) * kTZ;
    const int b = blockIdx.y;
    const int lx = threadIdx.x % kTX, ly = (threadIdx.x / kTX) % kTY, lz = threadIdx.x / (kTX * kTY);
    const size_t grid_nodes = (size_t)d.D * d.H * d.W;
    const float *inb = in + (size_t)b * grid_nodes * cin;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.0f;
    for (int c0 = 0; c0 < cin; c0 += kCK) {
        const int ck = min(kCK, cin - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < kHalo * ck; e += kConvThreads) {
            const int node = e / ck, c = e - node * ck;
            const int hx = node % kHX, hy = (node / kHX) % kHY, hz = node / (kHX * kHY);
            const int z = z0 + hz - 1, y = y0 + hy - 1, x = x0 + hx - 1;
            float v = 0.0f;
            if (z >= 0 && z < d.D && y >= 0 && y < d.H && x >= 0 && x < d.W) {
                v = inb[(((size_t)z * d.H + y) * d.W + x) * cin + c0 + c];
                if (relu_in) v = fmaxf(v, 0.0f);
            }
            s_in[node * (kCK + 1) + c] = v;
        }
        for (int e = threadIdx.x; e < 27 * ck * COUT; e += kConvThreads) {
            const int t = e / (ck * COUT), r = e - t * ck * COUT;  // r = c * COUT + co
            s_w[t * kCK * COUT + r] = w[((size_t)t * cin + c0) * COUT + r];
        }
        __syncthreads();
        for (int t = 0; t < 27; ++t) {
            const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
            const float *xv = s_in + (((lz + dz) * kHY + (ly + dy)) * kHX + (lx + dx)) * (kCK + 1);
            const float *wt = s_w + t * kCK * COUT;
            for (int c = 0; c < ck; ++c) {
                const float v = xv[c];
#pragma unroll
                for (int co = 0; co < COUT; ++co) acc[co] = fmaf(v, wt[c * COUT + co], acc[co]);
            }
        }
    }
    const int z = z0 + lz, y = y0 + ly, x = x0 + lx;
    if (z < d.D && y < d.H && x < d.W) {
        const size_t o = ((size_t)b * grid_nodes + ((size_t)z * d.H + y) * d.W + x) * COUT;
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            float v = acc[co];
            if (gate && !(gate[o + co] > 0.0f)) v = 0.0f;
            out[o + co] = v;
        }
    }
}

// Weight gradient, stage 1. Block (r, t): taps t < 27 accumulate
// sum_p act(in[p + off(t)][ci]) dy[p][co] over the positions of chunks r, r + R, ...;
// t = 27 accumulates sum_p dy[p][co] (the bias). Chunks are 128 consecutive positions.
constexpr int kWgThreads = 256, kWgChunk = 128;

template <int COUT>
__global__ void __launch_bounds__(kWgThreads)
    conv3d_wgrad_kernel(ConvDims d, int cin, const float *__restrict__ in, int relu_in,
                        const float *__restrict__ dy, float *__restrict__ partial) {
    __shared__ float s_x[kWgChunk * 33];
    __shared__ float s_dy[kWgChunk * COUT];
    const int r = blockIdx.x, R = gridDim.x, t = blockIdx.y;
    const bool is_bias = t == 27;
    const int rows = is_bias ? 1 : cin;
    const int E = rows * COUT;                 // entries of this tap
    const int dz = t / 9 - 1, dyo = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const long long grid_nodes = (long long)d.D * d.H * d.W;
    const long long chunks_per_grid = (grid_nodes + kWgChunk - 1) / kWgChunk;
    const long long chunks = chunks_per_grid * d.nb;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // entries threadIdx.x + 256 k
    for (long long ch = r; ch < chunks; ch += R) {
        const int b = (int)(ch / chunks_per_grid);
        const long long p0 = (ch - (long long)b * chunks_per_grid) * kWgChunk;
        const int np = (int)min((long long)kWgChunk, grid_nodes - p0);
        __syncthreads();
        for (int e = threadIdx.x; e < kWgChunk * COUT; e += kWgThreads) {
            const int q = e / COUT;
            s_dy[e] = q < np ? dy[((size_t)b * grid_nodes + p0 + q) * COUT + (e - q * COUT)] : 0.0f;
        }
        if (!is_bias) {
            for (int e = threadIdx.x; e < kWgChunk * cin; e += kWgThreads) {
                const int q = e / cin, c = e - q * cin;
                float v = 0.0f;
                if (q < np) {
                    const long long p = p0 + q;
                    const int x = (int)(p % d.W);
                    const long long zy = p / d.W;
                    const int y = (int)(zy % d.H), z = (int)(zy / d.H);
                    const int zz = z + dz, yy = y + dyo, xx = x + dx;
                    if (zz >= 0 && zz < d.D && yy >= 0 && yy < d.H && xx >= 0 && xx < d.W) {
                        v = in[((size_t)b * grid_nodes + ((size_t)zz * d.H + yy) * d.W + xx) * cin + c];
                        if (relu_in) v = fmaxf(v, 0.0f);
                    }
                }
                s_x[q * 33 + c] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = threadIdx.x + k * kWgThreads;
            if (e >= E) break;
            const int ci = e / COUT, co = e - ci * COUT;
            float a = acc[k];
            if (is_bias) {
                for (int q = 0; q < np; ++q) a += s_dy[q * COUT + co];
            } else {
                for (int q = 0; q < np; ++q) a = fmaf(s_x[q * 33 + ci], s_dy[q * COUT + co], a);
            }
            acc[k] = a;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int e = threadIdx.x + k * kWgThreads;
        if (e < E) partial[((size_t)r * 28 + t) * 1024 + e] = acc[k];
    }
}

// Weight gradient, stage 2: fixed-order sum over the R partial rows.
__global__ void wgrad_reduce_kernel(int cin, int cout, int R, const float *__restrict__ partial,
                                    float *__restrict__ gw, float *__restrict__ gb) {
    const int nw = 27 * cin * cout;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nw + cout) return;
    int t, idx;
    if (e < nw) {
        t = e / (cin * cout);
        idx = e - t * cin * cout;
    } else {
        t = 27;
        idx = e - nw;
    }
    double s = 0.0;
    for (int r = 0; r < R; ++r) s += partial[((size_t)r * 28 + t) * 1024 + idx];
    if (e < nw) gw[e] = (float)s;
    else gb[idx] = (float)s;
}

__global__ void flip_kernel(int cin, int cout, const float *__restrict__ w, float *__restrict__ wt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 27 * cin * cout) return;
    const int t = e / (cin * cout), r = e - t * cin * cout;
    const int ci = r / cout, co = r - ci * cout;
    wt[((size_t)(26 - t) * cout + co) * cin + ci] = w[e];
}

// Masked squared error, stage 1: per-block sums of mask and mask * (y - t)^2.
constexpr int kMseBlocks = 1024, kMseThreads = 256;

__global__ void __launch_bounds__(kMseThreads)
    mse_partial_kernel(long long total, const float *__restrict__ y, const float *__restrict__ tg,
                       const float *__restrict__ m, double *__restrict__ scratch) {
    __shared__ double s_a[kMseThreads], s_b[kMseThreads];
    double a = 0.0, c = 0.0;
    for (long long q = (long long)blockIdx.x * kMseThreads + threadIdx.x; q < total;
         q += (long long)gridDim.x * kMseThreads) {
        const double r = (double)y[q] - ((double)tg[q] - 1.0);  // target tau - 1
        a += m[q];
        c += m[q] * r * r;
    }
    s_a[threadIdx.x] = a;
    s_b[threadIdx.x] = c;
    __syncthreads();
    for (int h = kMseThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s_a[threadIdx.x] += s_a[threadIdx.x + h];
            s_b[threadIdx.x] += s_b[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = s_a[0];
        scratch[kMseBlocks + blockIdx.x] = s_b[0];
    }
}

// Stage 2 (one thread, fixed order): loss and 1 / sum(mask) into scratch[2 * kMseBlocks].
__global__ void mse_final_kernel(double *__restrict__ scratch, double *__restrict__ loss) {
    double a = 0.0, c = 0.0;
    for (int q = 0; q < kMseBlocks; ++q) {
        a += scratch[q];
        c += scratch[kMseBlocks + q];
    }
    const double inv = a > 0.0 ? 1.0 / a : 0.0;
    *loss = c * inv;
    scratch[2 * kMseBlocks] = inv;
}

__global__ void mse_grad_kernel(long long total, const float *__restrict__ y,
                                const float *__restrict__ tg, const float *__restrict__ m,
                                const double *__restrict__ scratch, float *__restrict__ dy) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= total) return;
    const double inv = scratch[2 * kMseBlocks];
    dy[q] = (float)(2.0 * (double)m[q] * ((double)y[q] - ((double)tg[q] - 1.0)) * inv);
}

__global__ void adam_kernel(int n, float *__restrict__ th, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.0f - b1) * gi;
    const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    th[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <typename F>
__global__ void features_kernel(GridC g, NetGrid ng, int B, int b0, int nb,
                                const SrcC *__restrict__ src,
                                const Vec2<F> *__restrict__ tabT, const Vec2<F> *__restrict__ tabP,
                                const F *__restrict__ rad, const F *__restrict__ cost,
                                const F *__restrict__ s, const F *__restrict__ xi,
                                const F *__restrict__ eta, float *__restrict__ x) {
    const long long Nn = (long long)ng.nr * ng.nt * ng.np;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Nn * nb) return;
    const int bl = (int)(q / Nn);
    const long long nn = q - (long long)bl * Nn;
    const int b = b0 + bl;
    // node of the network grid -> node of the solver grid
    const int kc = (int)(nn % ng.np);
    const long long tq = nn / ng.np;
    const int jc = (int)(tq % ng.nt), ic = (int)(tq / ng.nt);
    const int i = min(ic * ng.c, g.nr - 1), j = min(jc * ng.c, g.nt - 1),
              k = min(kc * ng.c, g.np - 1);
    const long long n = node_index(g, i, j, k);
    const SrcReg<F> S = load_src<F>(src, b, g.dr);
    F du, dn, de;
    source_offset<F>(S, i, rad[i], cost[j], tabT[(long long)j * B + b], tabP[(long long)k * B + b],
                     g.flat != 0, du, dn, de);
    float *o = x + q * kNetFeatures;
    o[0] = (float)(s[n] * S.inv_s0 - (F)1);
    o[1] = (float)xi[n];
    o[2] = (float)eta[n];
    o[3] = (float)du / kNetFeatureScaleKm;
    o[4] = (float)dn / kNetFeatureScaleKm;
    o[5] = (float)de / kNetFeatureScaleKm;
}

template <typename F>
__global__ void warm_tau_kernel(long long N, int B, int b0, int nb, const float *__restrict__ y,
                                F *__restrict__ tau) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N * nb) return;
    const int bl = (int)(q % nb);
    const long long n = q / nb;
    // a NaN prediction starts the node at tau = 1; the others (+-inf included) are clamped
    const float yv = y[(long long)bl * N + n];
    const float v = yv == yv ? fminf(fmaxf(yv, kNetClampLo), kNetClampHi) : 0.0f;
    tau[n * B + b0 + bl] = (F)(1.0f + v);
}

// Position of a node of the solver grid within the network grid along one axis: the lower
// network node a and the weight f of the upper one (network node a sits at min(a c, n - 1)).
__device__ __forceinline__ void net_axis_pos(int i, int c, int nc, int n, int &a, float &f) {
    a = min(i / c, nc - 2);
    const int p0 = a * c, p1 = min(p0 + c, n - 1);
    f = (float)(i - p0) / (float)(p1 - p0);
}

// tau = 1 + the trilinear interpolation of clamp(y) from the network grid (a NaN prediction
// counts as 0), for the network-grid stride ng.c > 1.
template <typename F>
__global__ void warm_tau_up_kernel(GridC g, NetGrid ng, int B, int b0, int nb,
                                   const float *__restrict__ y, F *__restrict__ tau) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= g.N * nb) return;
    const int bl = (int)(q % nb);
    const long long n = q / nb;
    const int k = (int)(n % g.np);
    const long long tq = n / g.np;
    const int j = (int)(tq % g.nt), i = (int)(tq / g.nt);
    int a[3];
    float f[3];
    net_axis_pos(i, ng.c, ng.nr, g.nr, a[0], f[0]);
    net_axis_pos(j, ng.c, ng.nt, g.nt, a[1], f[1]);
    net_axis_pos(k, ng.c, ng.np, g.np, a[2], f[2]);
    const float *yb = y + (long long)bl * ng.nr * ng.nt * ng.np;
    float v = 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int di = u >> 2, dj = (u >> 1) & 1, dk = u & 1;
        const float w = (di ? f[0] : 1.0f - f[0]) * (dj ? f[1] : 1.0f - f[1]) *
                        (dk ? f[2] : 1.0f - f[2]);
        const float yv = yb[((long long)(a[0] + di) * ng.nt + a[1] + dj) * ng.np + a[2] + dk];
        const float c = yv == yv ? fminf(fmaxf(yv, kNetClampLo), kNetClampHi) : 0.0f;
        v = fmaf(w, c, v);
    }
    tau[n * B + b0 + bl] = (F)(1.0f + v);
}

__global__ void round_bf16_kernel(int n, const float *__restrict__ in, float *__restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = __bfloat162float(__float2bfloat16_rn(in[e]));
}

inline unsigned blocks_of(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t run_conv3d(const ConvDims &d, int cin, int cout, const float *in, bool relu_in,
                       const float *w, const float *bias, const float *gate, float *out,
                       cudaStream_t st) {
    const int tiles = ((d.W + kTX - 1) / kTX) * ((d.H + kTY - 1) / kTY) * ((d.D + kTZ - 1) / kTZ);
    dim3 grid(tiles, d.nb);
    if (cout == 32)
        conv3d_kernel<32><<<grid, kConvThreads, 0, st>>>(d, cin, in, relu_in, w, bias, gate, out);
    else if (cout == 1)
        conv3d_kernel<1><<<grid, kConvThreads, 0, st>>>(d, cin, in, relu_in, w, bias, gate, out);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t run_conv3d_wgrad(const ConvDims &d, int cin, int cout, const float *in,
                             bool relu_in, const float *dy, float *partial, float *gw,
                             float *gb, cudaStream_t st) {
    if (cin > 32 || cin * cout > 1024) return cudaErrorInvalidValue;
    dim3 grid(kWgradBlocks, 28);
    if (cout == 32)
        conv3d_wgrad_kernel<32><<<grid, kWgThreads, 0, st>>>(d, cin, in, relu_in, dy, partial);
    else if (cout == 1)
        conv3d_wgrad_kernel<1><<<grid, kWgThreads, 0, st>>>(d, cin, in, relu_in, dy, partial);
    else
        return cudaErrorInvalidValue;
    const int n = 27 * cin * cout + cout;
    wgrad_reduce_kernel<<<blocks_of(n, 256), 256, 0, st>>>(cin, cout, kWgradBlocks, partial, gw, gb);
    return cudaGetLastError();
}

cudaError_t run_wgrad_reduce(int cin, int cout, int parts, const float *partial, float *gw,
                             float *gb, cudaStream_t st) {
    if (parts < 1 || parts > kWgradBlocks || cin * cout > 1024) return cudaErrorInvalidValue;
    const int n = 27 * cin * cout + cout;
    wgrad_reduce_kernel<<<blocks_of(n, 256), 256, 0, st>>>(cin, cout, parts, partial, gw, gb);
    return cudaGetLastError();
}

cudaError_t run_conv3d_flip(int cin, int cout, const float *w, float *wt, cudaStream_t st) {
    flip_kernel<<<blocks_of(27 * cin * cout, 256), 256, 0, st>>>(cin, cout, w, wt);
    return cudaGetLastError();
}

cudaError_t run_mse(long long total, const float *y, const float *target, const float *mask,
                    float *dy, double *scratch, double *loss, cudaStream_t st) {
    mse_partial_kernel<<<kMseBlocks, kMseThreads, 0, st>>>(total, y, target, mask, scratch);
    mse_final_kernel<<<1, 1, 0, st>>>(scratch, loss);
    mse_grad_kernel<<<blocks_of(total, 256), 256, 0, st>>>(total, y, target, mask, scratch, dy);
    return cudaGetLastError();
}

cudaError_t run_adam(int n, float *theta, const float *grad, float *m, float *v, int step,
                     float lr, float beta1, float beta2, float eps, cudaStream_t st) {
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    adam_kernel<<<blocks_of(n, 256), 256, 0, st>>>(n, theta, grad, m, v, lr, beta1, beta2, eps, c1, c2);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_net_features(const GridC &g, const NetGrid &ng, int B, int b0, int nb,
                             const SrcC *src, const Vec2<F> *tabT, const Vec2<F> *tabP,
                             const F *rad, const F *cost, const F *s, const F *xi, const F *eta,
                             float *x, cudaStream_t st) {
    const long long Nn = (long long)ng.nr * ng.nt * ng.np;
    features_kernel<F><<<blocks_of(Nn * nb, 256), 256, 0, st>>>(g, ng, B, b0, nb, src, tabT, tabP,
                                                                rad, cost, s, xi, eta, x);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_warm_tau(const GridC &g, const NetGrid &ng, int B, int b0, int nb,
                         const float *y, F *tau, cudaStream_t st) {
    if (ng.c == 1)
        warm_tau_kernel<F><<<blocks_of(g.N * nb, 256), 256, 0, st>>>(g.N, B, b0, nb, y, tau);
    else
        warm_tau_up_kernel<F><<<blocks_of(g.N * nb, 256), 256, 0, st>>>(g, ng, B, b0, nb, y, tau);
    return cudaGetLastError();
}

cudaError_t run_round_bf16(int n, const float *in, float *out, cudaStream_t st) {
    round_bf16_kernel<<<blocks_of(n, 256), 256, 0, st>>>(n, in, out);
    return cudaGetLastError();
}

#define TTGB_NET_INST(F)                                                                      \
    template cudaError_t run_net_features<F>(const GridC &, const NetGrid &, int, int, int,    \
                                             const SrcC *, const Vec2<F> *, const Vec2<F> *,  \
                                             const F *, const F *, const F *, const F *,      \
                                             const F *, float *, cudaStream_t);               \
    template cudaError_t run_warm_tau<F>(const GridC &, const NetGrid &, int, int, int,       \
                                         const float *, F *, cudaStream_t);
TTGB_NET_INST(float)
TTGB_NET_INST(double)
#undef TTGB_NET_INST

}  // namespace ttgb
