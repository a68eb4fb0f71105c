// Set-up and non-sweep kernels of libttgb: per-source factor constants, per-node model
// records, the T = T0 tau output, receiver interpolation tables, the misfit and adjoint
// sources (Eqs. 2-3, A2-A3), the point-source term of Eq. 5 and the kernel accumulation
// (Eqs. 6-8).
#include <cuda_runtime.h>

#include "tt_aux.h"

namespace ttgb {

namespace {

template <typename F> __device__ inline double ld_model(const F *p, long long n) {
    return (double)__ldg(p + n);
}

// Trilinear cell of a point (in fractional grid indices): base corner and 8 weights, corner
// c = di*4 + dj*2 + dk.
__device__ inline void cell_of(const GridC &g, double fr, double ft, double fp, int base[3],
                               double w[8]) {
    double f[3] = {fr, ft, fp};
    int n[3] = {g.nr, g.nt, g.np};
    double u[3];
    for (int a = 0; a < 3; ++a) {
        int i0 = (int)floor(f[a]);
        i0 = i0 < 0 ? 0 : (i0 > n[a] - 2 ? n[a] - 2 : i0);
        base[a] = i0;
        u[a] = f[a] - i0;
    }
    for (int c = 0; c < 8; ++c) {
        double wr = (c & 4) ? u[0] : 1.0 - u[0];
        double wt = (c & 2) ? u[1] : 1.0 - u[1];
        double wp = (c & 1) ? u[2] : 1.0 - u[2];
        w[c] = wr * wt * wp;
    }
}

__device__ inline long long corner_node(const GridC &g, const int base[3], int c) {
    return node_index(g, base[0] + ((c >> 2) & 1), base[1] + ((c >> 1) & 1), base[2] + (c & 1));
}

__device__ inline void frac_of(const GridC &g, const PointD &p, double &fr, double &ft,
                               double &fp) {
    const double deg = 3.14159265358979323846 / 180.0;
    fr = ((g.re - p.depth) - g.r0) / g.dr;
    ft = (p.lat * deg - g.t0) / g.dt;
    fp = (p.lon * deg - g.p0) / g.dp;
}

// One thread per source: interpolated (s0, xi0, eta0), M0^-1, frame sines, fixed set.
template <typename F>
__global__ void source_setup_kernel(GridC g, const F *s, const F *xi, const F *eta,
                                    const PointD *pts, int n_src, SrcC *out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_src) return;
    SrcC S;
    frac_of(g, pts[b], S.fr, S.ft, S.fp);
    int base[3];
    double w[8];
    cell_of(g, S.fr, S.ft, S.fp, base, w);
    double s0 = 0, x0 = 0, e0 = 0;
    for (int c = 0; c < 8; ++c) {
        long long n = corner_node(g, base, c);
        s0 += w[c] * ld_model(s, n);
        x0 += w[c] * ld_model(xi, n);
        e0 += w[c] * ld_model(eta, n);
    }
    double det = (1.0 - 2.0 * x0) * (1.0 + 2.0 * x0) - 4.0 * e0 * e0;
    S.b11 = (1.0 + 2.0 * x0) / det;
    S.b12 = -2.0 * e0 / det;
    S.b22 = (1.0 - 2.0 * x0) / det;
    S.s0 = s0;
    S.inv_s0 = 1.0 / s0;
    const double deg = 3.14159265358979323846 / 180.0;
    S.sts = sin(pts[b].lat * deg);
    S.cts = cos(pts[b].lat * deg);
    S.ir = (int)floor(S.fr);
    S.frr = S.fr - S.ir;
    int n[3] = {g.nr, g.nt, g.np};
    double f[3] = {S.fr, S.ft, S.fp};
    int c3[3];
    for (int a = 0; a < 3; ++a) {
        int c = (int)floor(f[a] + 0.5);
        c3[a] = c < 0 ? 0 : (c > n[a] - 1 ? n[a] - 1 : c);
    }
    S.ci = c3[0]; S.cj = c3[1]; S.ck = c3[2];
    out[b] = S;
}

// Angle tables per (latitude row or longitude column, source): (sin d, 1 - cos d) with
// d = (index - f_source) * spacing, or (R_E d, 0) in the flat geometry. Layout [row][source].
template <typename F>
__global__ void angle_table_kernel(GridC g, const SrcC *S, int n_src, int axis, Vec2<F> *tab) {
    int n_rows = axis == 1 ? g.nt : g.np;
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)n_rows * n_src) return;
    int row = (int)(q / n_src), b = (int)(q % n_src);
    double f = axis == 1 ? S[b].ft : S[b].fp;
    double h = axis == 1 ? g.dt : g.dp;
    double d = ((double)row - f) * h;
    Vec2<F> v;
    if (g.flat) {
        v.x = (F)(g.re * d);
        v.y = (F)0;
    } else {
        double sh = sin(0.5 * d);
        v.x = (F)sin(d);
        v.y = (F)(2.0 * sh * sh);
    }
    tab[q] = v;
}

// Per-node record of the forward sweep (s, xi, eta and the Lax-Friedrichs coefficients).
template <typename F>
__global__ void node_record_kernel(GridC g, const F *s, const F *xi, const F *eta,
                                   const double *h2, const double *cost, NodeRec<F> *rec,
                                   int *bad) {
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    long long t = n / g.np;
    int j = (int)(t % g.nt);
    int i = (int)(t / g.nt);
    double sv = ld_model(s, n), xv = ld_model(xi, n), ev = ld_model(eta, n);
    // bit 0: an invalid model; bit 1: an anisotropic node (refused by the Godunov solver)
    if (!(sv > 0.0) || !(xv * xv + ev * ev < 0.25)) atomicOr(bad, 1);
    if (xv != 0.0 || ev != 0.0) atomicOr(bad, 2);
    double er = 0.5 / g.dr;
    double et = 0.5 / (g.dt * h2[i]);
    double ep = 0.5 / (g.dp * h2[i] * cost[j]);
    double kt = sqrt(fmax(1.0 - 2.0 * xv, 0.0)), kp = sqrt(fmax(1.0 + 2.0 * xv, 0.0));
    NodeRec<F> R;
    R.s = (F)sv; R.xi = (F)xv; R.eta = (F)ev;
    R.ct = (F)(kt * et); R.cp = (F)(kp * ep);
    R.invW = (F)(0.5 / (er + kt * et + kp * ep));
    R.et = (F)et; R.ep = (F)ep;
    rec[n] = R;
}

template <typename F>
__global__ void fill_kernel(F *p, long long n, F v) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) p[q] = v;
}

// tau = 1 on each source's 3x3x3 fixed set (Sec. 3.1: T = T0 there).
template <typename F>
__global__ void fix_set_kernel(GridC g, const SrcC *S, int n_src, F *tau) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_src * 27) return;
    int b = q / 27, c = q % 27;
    int i = S[b].ci + c / 9 - 1, j = S[b].cj + (c / 3) % 3 - 1, k = S[b].ck + c % 3 - 1;
    if (i < 0 || j < 0 || k < 0 || i >= g.nr || j >= g.nt || k >= g.np) return;
    tau[node_index(g, i, j, k) * n_src + b] = (F)1;
}

// Start from above (opts.init = 3). The fast sweeping method starts from large values
// outside the fixed set, so that the upwind (Godunov) update only lowers them toward the
// solution. The value used is twice a bound of tau. Along the straight ray of length L from
// the source, T <= max_ray(s N) L, where N(d) = sqrt(d^T M^-1 d) is the direction factor of
// the local metric M of the Hamiltonian (eigenvalues 1 and 1 +- 2 g, g = sqrt(xi^2 + eta^2)).
// The factor is T0 = s0 N0(d) L, so tau <= hi / lo with
//   hi = max_n s_n / sqrt(1 - 2 g_n),   lo = min_n s_n / sqrt(1 + 2 g_n).
// The factor 2 leaves room for the discretisation error. Where the start is not above the
// solution the sweep still reaches the same fixed point, only in more iterations.
// hilo[0] and hilo[1] hold hi and lo as the bits of positive floats (their unsigned order is
// the float order); the caller sets them to 0 and to a large float first.
template <typename F>
__global__ void upper_bound_kernel(long long N, const F *s, const F *xi, const F *eta,
                                   unsigned *hilo) {
    float hi = 0.f, lo = 3.0e38f;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const float sv = (float)s[n], a = (float)xi[n], b = (float)eta[n];
        const float g2 = sqrtf(a * a + b * b) * 2.f;
        if (sv > 0.f) {
            hi = fmaxf(hi, sv / sqrtf(fmaxf(1.f - g2, 1e-6f)));
            lo = fminf(lo, sv / sqrtf(1.f + g2));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    }
    __shared__ float shi[32], slo[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        shi[w] = hi;
        slo[w] = lo;
    }
    __syncthreads();
    if (w == 0) {
        hi = lane < nw ? shi[lane] : 0.f;
        lo = lane < nw ? slo[lane] : 3.0e38f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        }
        if (lane == 0) {
            atomicMax(hilo, __float_as_uint(hi));
            atomicMin(hilo + 1, __float_as_uint(lo));
        }
    }
}

template <typename F>
__global__ void upper_fill_kernel(F *tau, long long n, const unsigned *hilo) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float hi = __uint_as_float(hilo[0]), lo = __uint_as_float(hilo[1]);
    tau[q] = (F)(2.f * hi / lo);
}

// Batch order of a plan's forward sweep. The sweep's barrier groups take consecutive sources
// of the batch; ordered by their previous forward iteration counts, a group holds sources that
// converge together and retires early instead of holding its SMs for one slow source. perm[q]
// is the source at position q of the ordered batch. Each source's arithmetic does not depend
// on its position, so the results are the same bits in any order.
__global__ void gather_points_kernel(int B, const int *__restrict__ perm,
                                     const PointD *__restrict__ in, PointD *__restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < B) out[q] = in[perm[q]];
}

// tau_o[n][q] = tau[n][perm[q]] (to_order) or tau[n][perm[q]] = tau_o[n][q] (back); rows of B.
template <typename F>
__global__ void permute_rows_kernel(long long N, int B, const int *__restrict__ perm,
                                    F *__restrict__ tau, F *__restrict__ tau_o, bool to_order) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N * B) return;
    const long long n = x / B;
    const int q = (int)(x - n * B);
    const long long y = n * B + perm[q];
    if (to_order) tau_o[x] = tau[y];
    else tau[y] = tau_o[x];
}

// out[q][c] = in[perm[q]][c] for rows of n doubles (a batch's receiver residuals, ordered).
__global__ void gather_rows_kernel(int B, int n, const int *__restrict__ perm,
                                  const double *__restrict__ in, double *__restrict__ out) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= (long long)B * n) return;
    const int q = (int)(x / n), c = (int)(x - (long long)q * n);
    out[x] = in[(long long)perm[q] * n + c];
}

__global__ void unpermute_ints_kernel(int B, const int *__restrict__ perm,
                                      const int *__restrict__ a_o, const int *__restrict__ b_o,
                                      int *__restrict__ a, int *__restrict__ b) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B) return;
    a[perm[q]] = a_o[q];
    b[perm[q]] = b_o[q];
}

// perm = the sources sorted by (iterations, index), ascending: the rank of source i is the
// number of sources before it in that order. One block; O(B^2) comparisons (B <= 4096).
__global__ void order_by_iterations_kernel(int B, const int *__restrict__ iters,
                                           int *__restrict__ perm) {
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const int ti = iters[i];
        int rank = 0;
        for (int j = 0; j < B; ++j) {
            const int tj = iters[j];
            rank += tj < ti || (tj == ti && j < i);
        }
        perm[rank] = i;
    }
}

__global__ void identity_kernel(int B, int *__restrict__ perm) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < B) perm[q] = q;
}

// T = T0 tau at every (node, source).
template <typename F>
__global__ void traveltime_kernel(GridC g, int B, const SrcC *src, const Vec2<F> *tabT,
                                  const Vec2<F> *tabP, const F *rad, const F *cost,
                                  const F *sint, const F *tau, F *T) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= g.N * B) return;
    int b = (int)(q % B);
    long long n = q / B;
    int k = (int)(n % g.np);
    long long t = n / g.np;
    int j = (int)(t % g.nt);
    int i = (int)(t / g.nt);
    SrcReg<F> S = load_src<F>(src, b, g.dr);
    F ur, ut, up;
    F invT0 = factor_T0<F>(S, i, rad[i], cost[j], sint[j], tabT[(long long)j * B + b],
                           tabP[(long long)k * B + b], g.flat != 0, ur, ut, up);
    // invT0 is infinite only at a node that coincides with the source, where T0 = 0.
    T[q] = isinf(invT0) ? (F)0 : tau[q] / invT0;
}

// Receiver cells: for receiver m, corner q = 8 m + c has node cq[q], trilinear weight wq[q].
__global__ void receiver_setup_kernel(GridC g, const PointD *rec, int n_rec, long long *cq,
                                      double *wq, int *bad) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_rec) return;
    double fr, ft, fp;
    frac_of(g, rec[m], fr, ft, fp);
    const double eps = 1e-9;
    if (!(fr >= -eps && fr <= g.nr - 1 + eps && ft >= -eps && ft <= g.nt - 1 + eps &&
          fp >= -eps && fp <= g.np - 1 + eps))
        atomicExch(bad, 1);
    int base[3];
    double w[8];
    cell_of(g, fr, ft, fp, base, w);
    for (int c = 0; c < 8; ++c) {
        cq[8 * m + c] = corner_node(g, base, c);
        wq[8 * m + c] = w[c];
    }
}

// Chain of receiver corners sharing a node, in increasing corner order: head = smallest q.
__global__ void corner_head_kernel(const long long *cq, int S, int *sidx) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < S) atomicMin(&sidx[cq[q]], q);
}

__global__ void corner_next_kernel(const long long *cq, int S, int *next) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= S) return;
    int nx = kNone;
    for (int r = q + 1; r < S; ++r)
        if (cq[r] == cq[q]) { nx = r; break; }
    next[q] = nx;
}

__global__ void corner_compact_kernel(const long long *cq, int S, const int *sidx, int *heads,
                                      int *n_heads) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < S && sidx[cq[q]] == q) heads[atomicAdd(n_heads, 1)] = q;
}

__global__ void corner_relabel_kernel(const long long *cq, const int *heads, const int *n_heads,
                                      int *sidx) {
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < *n_heads) sidx[cq[heads[h]]] = h;
}

// J_c S_c of Eq. 5 at every node that holds a receiver corner, per source:
// sum over the node's corners (in corner order) of R[b][m] w / (dr dt dp), in FP64.
template <typename F>
__global__ void point_source_kernel(const int *heads, const int *n_heads, const int *next,
                                    const double *wq, const double *R, int n_rec, int B,
                                    double inv_vol, F *JS) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)(*n_heads) * B) return;
    int h = (int)(q / B), b = (int)(q % B);
    double acc = 0.0;
    for (int c = heads[h]; c != kNone; c = next[c])
        acc += R[(long long)b * n_rec + c / 8] * wq[c] * inv_vol;
    JS[q] = (F)acc;
}

// Misfit of one source per warp. Lanes own receivers m = lane (mod 32); every record is
// applied by the owner lanes in record order, so the adjoint sources are bitwise
// reproducible. Dynamic shared memory: per warp, Tr[n_rec] and R[n_rec] in double.
// TABLE = false: the receiver times are interpolated from the fields T (cq, wq);
// TABLE = true: they are given, Tr[b][m] = tab[b][m] + otime[b] (otime may be NULL).
template <typename F, bool TABLE>
__global__ void misfit_kernel(int B, int n_rec, const F *T, const long long *cq,
                              const double *wq, const double *tab, const double *otime,
                              const int *abs_off, const int *abs_rec,
                              const double *abs_tobs, const double *abs_w, const int *cs_off,
                              const int *cs_m, const int *cs_i, const double *cs_dtobs,
                              const double *cs_w, double alpha, double beta, double *Tr_out,
                              double *chi_out, double *R_out, int *bad) {
    extern __shared__ double sh[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= B) return;
    double *Tr = sh + (size_t)warp * 2 * n_rec;
    double *R = Tr + n_rec;
    const double t0 = TABLE && otime ? otime[b] : 0.0;
    for (int m = lane; m < n_rec; m += 32) {
        double acc = 0.0;
        if (TABLE) {
            acc = tab[(long long)b * n_rec + m] + t0;
        } else {
            for (int c = 0; c < 8; ++c)
                acc += wq[8 * m + c] * (double)T[cq[8 * m + c] * B + b];
        }
        Tr[m] = acc;
        R[m] = 0.0;
        if (Tr_out) Tr_out[(long long)b * n_rec + m] = acc;
    }
    __syncwarp();
    double chi_t = 0.0, chi_cs = 0.0;
    // absolute times, Eq. 2 / A2
    const int a0 = abs_off[b], a1 = abs_off[b + 1];
    for (int base = a0; base < a1; base += 32) {
        int q = base + lane;
        int m = -1;
        double v = 0.0;
        if (q < a1) {
            m = abs_rec[q];
            if (m < 0 || m >= n_rec) { atomicExch(bad, 1); m = -1; }
            else {
                double e = Tr[m] - abs_tobs[q];
                chi_t += 0.5 * abs_w[q] * e * e;
                v = alpha * abs_w[q] * e;
            }
        }
        int cnt = min(32, a1 - base);
        for (int l = 0; l < cnt; ++l) {
            int ml = __shfl_sync(0xffffffffu, m, l);
            double vl = __shfl_sync(0xffffffffu, v, l);
            if (ml >= 0 && (ml & 31) == lane) R[ml] += vl;
        }
    }
    // common-source pairs, Eq. 3 / A3
    const int c0 = cs_off[b], c1 = cs_off[b + 1];
    for (int base = c0; base < c1; base += 32) {
        int q = base + lane;
        int m = -1, i = -1;
        double v = 0.0;
        if (q < c1) {
            m = cs_m[q];
            i = cs_i[q];
            if (m < 0 || m >= n_rec || i < 0 || i >= n_rec) { atomicExch(bad, 1); m = i = -1; }
            else {
                double e = (Tr[m] - Tr[i]) - cs_dtobs[q];
                chi_cs += 0.5 * cs_w[q] * e * e;
                v = beta * cs_w[q] * e;
            }
        }
        int cnt = min(32, c1 - base);
        for (int l = 0; l < cnt; ++l) {
            int ml = __shfl_sync(0xffffffffu, m, l);
            int il = __shfl_sync(0xffffffffu, i, l);
            double vl = __shfl_sync(0xffffffffu, v, l);
            if (ml >= 0 && (ml & 31) == lane) R[ml] += vl;
            if (il >= 0 && (il & 31) == lane) R[il] -= vl;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        chi_t += __shfl_xor_sync(0xffffffffu, chi_t, o);
        chi_cs += __shfl_xor_sync(0xffffffffu, chi_cs, o);
    }
    __syncwarp();
    for (int m = lane; m < n_rec; m += 32) R_out[(long long)b * n_rec + m] = R[m];
    if (lane == 0 && chi_out) {
        chi_out[2 * b] = chi_t;
        chi_out[2 * b + 1] = chi_cs;
    }
}

// Compensated accumulator of a lane's terms: (hi, lo) with hi + lo the sum to about twice
// the working precision (Knuth's TwoSum: hi + lo = old hi + term exactly, each step). In
// FP32 it keeps ~48 significant bits without the FP64 pipe, whose rate on this GPU is a
// small fraction of the FP32 rate; in FP64 it is plain double accumulation plus a
// correction word.
template <typename F> struct CompSum {
    F hi = 0, lo = 0;
    __device__ __forceinline__ void add(F x) {
        const F s = __fadd_rn_t(hi, x);
        const F bp = __fsub_rn_t(s, hi);
        const F err = __fadd_rn_t(__fsub_rn_t(hi, __fsub_rn_t(s, bp)), __fsub_rn_t(x, bp));
        hi = s;
        lo = __fadd_rn_t(lo, err);
    }
    // adds another accumulator's (hi, lo): TwoSum of the hi parts, the lo parts summed
    __device__ __forceinline__ void merge(F ohi, F olo) {
        add(ohi);
        lo = __fadd_rn_t(lo, olo);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    static __device__ __forceinline__ float __fadd_rn_t(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float __fsub_rn_t(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ double __fadd_rn_t(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double __fsub_rn_t(double a, double b) { return __dsub_rn(a, b); }
};

// Kernels of Eqs. 6-8, one warp per node; lanes stride over the sources and the warp sum
// runs in a fixed shuffle order.
template <typename F>
__global__ void kernel_accum_kernel(GridC g, int B, const F *s, const F *T, const F *P,
                                    const double *h2, const double *cost, double *Ks,
                                    double *Kxi, double *Keta) {
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    // Each source's term in the fields' precision F (its inputs are F values; reciprocals
    // instead of divisions). A lane sums its sources' terms with a compensated accumulator
    // in F (TwoSum), the warp merges the lanes' accumulators in a fixed butterfly, and lane 0
    // adds the batch's total to the FP64 kernels: only those three adds use the FP64 pipe.
    const F idt = (F)(1.0 / g.dt), idp = (F)(1.0 / g.dp);
    for (long long n = warp; n < g.N; n += nwarps) {
        int k = (int)(n % g.np);
        long long t = n / g.np;
        int j = (int)(t % g.nt);
        int i = (int)(t / g.nt);
        const F iht = (F)(1.0 / h2[i]), ihp = (F)(1.0 / (h2[i] * cost[j]));
        const F ct = iht * (j == 0 || j == g.nt - 1 ? idt : (F)0.5 * idt);
        const F cp = ihp * (k == 0 || k == g.np - 1 ? idp : (F)0.5 * idp);
        const long long st = (long long)g.np * B, sp = B;
        const long long ot_hi = j < g.nt - 1 ? st : 0, ot_lo = j > 0 ? st : 0;
        const long long op_hi = k < g.np - 1 ? sp : 0, op_lo = k > 0 ? sp : 0;
        CompSum<F> sP, sX, sE;
#pragma unroll 4
        for (int b = lane; b < B; b += 32) {
            const long long x = n * B + b;
            // central differences inside, one-sided on the faces (R10)
            const F gt = (T[x + ot_hi] - T[x - ot_lo]) * ct;
            const F gp = (T[x + op_hi] - T[x - op_lo]) * cp;
            const F p = P[x];
            sP.add(p);
            sX.add(p * (gt * gt - gp * gp));
            sE.add((F)-2 * p * gt * gp);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sP.merge(__shfl_xor_sync(0xffffffffu, sP.hi, o), __shfl_xor_sync(0xffffffffu, sP.lo, o));
            sX.merge(__shfl_xor_sync(0xffffffffu, sX.hi, o), __shfl_xor_sync(0xffffffffu, sX.lo, o));
            sE.merge(__shfl_xor_sync(0xffffffffu, sE.hi, o), __shfl_xor_sync(0xffffffffu, sE.lo, o));
        }
        if (lane == 0) {
            const double aP = sP.value(), aX = sX.value(), aE = sE.value();
            const double sv = (double)s[n];
            Ks[n] += sv * sv * aP;
            Kxi[n] += aX;
            Keta[n] += aE;
        }
    }
}

inline unsigned blocks_for(long long n, int threads) {
    return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

// ------------------------------------------------------------------------ host launchers

template <typename F>
cudaError_t run_source_setup(const GridC &g, const void *s, const void *xi, const void *eta,
                             const PointD *d_pts, int n_src, SrcC *d_src, Vec2<F> *tabT,
                             Vec2<F> *tabP, cudaStream_t st) {
    source_setup_kernel<F><<<blocks_for(n_src, 128), 128, 0, st>>>(
        g, (const F *)s, (const F *)xi, (const F *)eta, d_pts, n_src, d_src);
    angle_table_kernel<F><<<blocks_for((long long)g.nt * n_src, 256), 256, 0, st>>>(
        g, d_src, n_src, 1, tabT);
    angle_table_kernel<F><<<blocks_for((long long)g.np * n_src, 256), 256, 0, st>>>(
        g, d_src, n_src, 2, tabP);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_node_records(const GridC &g, const void *s, const void *xi, const void *eta,
                             const double *h2, const double *cost, NodeRec<F> *rec, int *bad,
                             cudaStream_t st) {
    node_record_kernel<F><<<blocks_for(g.N, 256), 256, 0, st>>>(
        g, (const F *)s, (const F *)xi, (const F *)eta, h2, cost, rec, bad);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_tau_init(const GridC &g, int n_src, const SrcC *d_src, F *tau, bool fill,
                         cudaStream_t st) {
    if (fill)
        fill_kernel<F><<<blocks_for(g.N * n_src, 256), 256, 0, st>>>(tau, g.N * n_src, (F)1);
    fix_set_kernel<F><<<blocks_for(27LL * n_src, 128), 128, 0, st>>>(g, d_src, n_src, tau);
    return cudaGetLastError();
}

cudaError_t run_order_identity(int B, int *perm, cudaStream_t st) {
    identity_kernel<<<blocks_for(B, 256), 256, 0, st>>>(B, perm);
    return cudaGetLastError();
}

cudaError_t run_order_update(int B, const int *iters, int *perm, cudaStream_t st) {
    order_by_iterations_kernel<<<1, 1024, 0, st>>>(B, iters, perm);
    return cudaGetLastError();
}

cudaError_t run_gather_points(int B, const int *perm, const PointD *in, PointD *out,
                              cudaStream_t st) {
    gather_points_kernel<<<blocks_for(B, 256), 256, 0, st>>>(B, perm, in, out);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_permute_rows(long long N, int B, const int *perm, F *tau, F *tau_o, bool to_order,
                             cudaStream_t st) {
    permute_rows_kernel<F><<<blocks_for(N * B, 256), 256, 0, st>>>(N, B, perm, tau, tau_o,
                                                                   to_order);
    return cudaGetLastError();
}

cudaError_t run_gather_rows(int B, int n, const int *perm, const double *in, double *out,
                            cudaStream_t st) {
    if (n > 0)
        gather_rows_kernel<<<blocks_for((long long)B * n, 256), 256, 0, st>>>(B, n, perm, in, out);
    return cudaGetLastError();
}

cudaError_t run_unpermute_ints(int B, const int *perm, const int *a_o, const int *b_o, int *a,
                               int *b, cudaStream_t st) {
    unpermute_ints_kernel<<<blocks_for(B, 256), 256, 0, st>>>(B, perm, a_o, b_o, a, b);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_upper_start(const GridC &g, int n_src, const void *s, const void *xi,
                            const void *eta, F *tau, unsigned *hilo, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(hilo, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(hilo + 1, 0x7f, sizeof(unsigned), st)) != cudaSuccess) return e;
    const unsigned nb = blocks_for(g.N, 256);
    upper_bound_kernel<F><<<nb < 1216u ? nb : 1216u, 256, 0, st>>>(
        g.N, (const F *)s, (const F *)xi, (const F *)eta, hilo);
    upper_fill_kernel<F><<<blocks_for(g.N * n_src, 256), 256, 0, st>>>(tau, g.N * n_src, hilo);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_traveltime(const GridC &g, int B, const SrcC *src, const Vec2<F> *tabT,
                           const Vec2<F> *tabP, const F *rad, const F *cost, const F *sint,
                           const F *tau, F *T, cudaStream_t st) {
    traveltime_kernel<F><<<blocks_for(g.N * B, 256), 256, 0, st>>>(g, B, src, tabT, tabP, rad,
                                                                   cost, sint, tau, T);
    return cudaGetLastError();
}

cudaError_t run_receiver_setup(const GridC &g, const PointD *d_rec, int n_rec, long long *cq,
                               double *wq, int *bad, cudaStream_t st) {
    receiver_setup_kernel<<<blocks_for(n_rec, 128), 128, 0, st>>>(g, d_rec, n_rec, cq, wq, bad);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_point_sources(const GridC &g, int n_rec, const long long *cq, const double *wq,
                              int *sidx, int *next, int *heads, int *n_heads, const double *R,
                              int B, F *JS, cudaStream_t st) {
    const int S = 8 * n_rec;
    cudaMemsetAsync(sidx, 0x7f, (size_t)g.N * sizeof(int), st);  // every entry = kNone
    cudaMemsetAsync(n_heads, 0, sizeof(int), st);
    corner_head_kernel<<<blocks_for(S, 256), 256, 0, st>>>(cq, S, sidx);
    corner_next_kernel<<<blocks_for(S, 256), 256, 0, st>>>(cq, S, next);
    corner_compact_kernel<<<blocks_for(S, 256), 256, 0, st>>>(cq, S, sidx, heads, n_heads);
    corner_relabel_kernel<<<blocks_for(S, 256), 256, 0, st>>>(cq, heads, n_heads, sidx);
    const double inv_vol = 1.0 / (g.dr * g.dt * g.dp);
    point_source_kernel<F><<<blocks_for((long long)S * B, 256), 256, 0, st>>>(
        heads, n_heads, next, wq, R, n_rec, B, inv_vol, JS);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_misfit(int B, int n_rec, const void *T, const long long *cq, const double *wq,
                       const tt_data &d, double *Tr, double *chi, double *R, int *bad,
                       cudaStream_t st) {
    const int warps = 4;
    size_t smem = (size_t)warps * 2 * n_rec * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(misfit_kernel<F, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    misfit_kernel<F, false><<<blocks_for(B, warps), warps * 32, smem, st>>>(
        B, n_rec, (const F *)T, cq, wq, nullptr, nullptr, d.d_abs_off, d.d_abs_rec, d.d_abs_tobs,
        d.d_abs_w, d.d_cs_off, d.d_cs_m, d.d_cs_i, d.d_cs_dtobs, d.d_cs_w, d.alpha, d.beta, Tr, chi,
        R, bad);
    return cudaGetLastError();
}

cudaError_t run_misfit_table(int B, int n_rec, const double *tab, const double *otime,
                             const tt_data &d, double *Tr, double *chi, double *R, int *bad,
                             cudaStream_t st) {
    const int warps = 4;
    size_t smem = (size_t)warps * 2 * n_rec * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(misfit_kernel<double, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    misfit_kernel<double, true><<<blocks_for(B, warps), warps * 32, smem, st>>>(
        B, n_rec, nullptr, nullptr, nullptr, tab, otime, d.d_abs_off, d.d_abs_rec, d.d_abs_tobs,
        d.d_abs_w, d.d_cs_off, d.d_cs_m, d.d_cs_i, d.d_cs_dtobs, d.d_cs_w, d.alpha, d.beta, Tr, chi,
        R, bad);
    return cudaGetLastError();
}

template <typename F>
cudaError_t run_kernel_accum(const GridC &g, int B, const void *s, const void *T, const void *P,
                             const double *h2, const double *cost, double *Ks, double *Kxi,
                             double *Keta, int n_sm, cudaStream_t st) {
    long long warps = g.N;
    long long cap = (long long)n_sm * 64;  // 64 warps per SM resident at most
    unsigned blocks = (unsigned)((warps < cap ? warps : cap) * 32 / 256);
    if (blocks == 0) blocks = 1;
    kernel_accum_kernel<F><<<blocks, 256, 0, st>>>(g, B, (const F *)s, (const F *)T,
                                                   (const F *)P, h2, cost, Ks, Kxi, Keta);
    return cudaGetLastError();
}

#define TTGB_INST(F)                                                                           \
    template cudaError_t run_source_setup<F>(const GridC &, const void *, const void *,        \
                                             const void *, const PointD *, int, SrcC *,        \
                                             Vec2<F> *, Vec2<F> *, cudaStream_t);              \
    template cudaError_t run_node_records<F>(const GridC &, const void *, const void *,        \
                                             const void *, const double *, const double *,     \
                                             NodeRec<F> *, int *, cudaStream_t);               \
    template cudaError_t run_tau_init<F>(const GridC &, int, const SrcC *, F *, bool,          \
                                         cudaStream_t);                                        \
    template cudaError_t run_permute_rows<F>(long long, int, const int *, F *, F *, bool,     \
                                             cudaStream_t);                                    \
    template cudaError_t run_upper_start<F>(const GridC &, int, const void *, const void *,    \
                                            const void *, F *, unsigned *, cudaStream_t);      \
    template cudaError_t run_traveltime<F>(const GridC &, int, const SrcC *, const Vec2<F> *,  \
                                           const Vec2<F> *, const F *, const F *, const F *,   \
                                           const F *, F *, cudaStream_t);                      \
    template cudaError_t run_point_sources<F>(const GridC &, int, const long long *,           \
                                              const double *, int *, int *, int *, int *,      \
                                              const double *, int, F *, cudaStream_t);         \
    template cudaError_t run_misfit<F>(int, int, const void *, const long long *,              \
                                       const double *, const tt_data &, double *, double *,    \
                                       double *, int *, cudaStream_t);                         \
    template cudaError_t run_kernel_accum<F>(const GridC &, int, const void *, const void *,   \
                                             const void *, const double *, const double *,     \
                                             double *, double *, double *, int, cudaStream_t);
TTGB_INST(float)
TTGB_INST(double)
#undef TTGB_INST

}  // namespace ttgb

namespace ttgb {

bool grid_constants(const tt_grid &G, GridC &g) {
    const int dims[3] = {G.n_r, G.n_t, G.n_p};
    for (int d : dims)
        if (d < 4 || d > TT_MAX_DIM) return false;
    if (!(G.depth_max_km > G.depth_min_km) || !(G.lat_max_deg > G.lat_min_deg) ||
        !(G.lon_max_deg > G.lon_min_deg) || !(G.earth_radius_km > G.depth_max_km))
        return false;
    if (G.geometry != TT_GEOM_SPHERICAL && G.geometry != TT_GEOM_FLAT) return false;
    if (G.geometry == TT_GEOM_SPHERICAL && (G.lat_min_deg <= -89.0 || G.lat_max_deg >= 89.0))
        return false;
    const double deg = 3.14159265358979323846 / 180.0;
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
    return true;
}

}  // namespace ttgb
