// Warm-start inference on the 5th-generation tensor cores: the four 3x3x3 convolutions of
// the network (tt_net.h) as implicit GEMMs issued with tcgen05.mma (BF16 operands, FP32
// accumulators in tensor memory), operands staged by TMA tensor copies.
//
// Row layout of the activations. The nodes of one grid are rows
//   r = (i (n_t + 1) + j) (n_p + 1) + k,   i < n_r, j <= n_t, k <= n_p,   r < R = n_r Si,
// of C BF16 channels (C = 16 for the input features, padded from 6; 32 for the hidden
// layers), the rows j = n_t and k = n_p being zero. A tap (di, dj, dk) of the convolution at
// row r reads row r + (di - 1) Si + (dj - 1) Sj + (dk - 1), with Sj = n_p + 1 and
// Si = (n_t + 1) Sj: every tap is a fixed row shift, the zero rows give the zero padding at
// the theta and phi faces, and rows outside [0, R) (the radial faces) are zero-filled by the
// tensor copy. Buffer [grid][R][C].
//
// GEMM of one tile: M = 128 consecutive rows r0 + m, K = 9 (di, dj) x C, and N = 3 x output
// channels: the three dk taps' weights side by side, so that the accumulator holds, for each
// dk, D_dk[m] = sum over (di, dj) of x[r0 + m + (di-1) Si + (dj-1) Sj - 1] W(di, dj, dk).
// Output row r0 + m is D_0[m] + D_1[m + 1] + D_2[m + 2]: the epilogue combines neighbouring
// TMEM lanes (warp shuffles, and a small shared-memory exchange across the four lane
// quarters), so a tile of 128 accumulator rows yields 126 outputs and the tiles step by 126
// rows. Every operand is thus an aligned block of whole rows, which lets both the A slabs
// (one TMA tensor copy of 128 rows per (di, dj)) and the weights use the swizzled K-major
// layout (64-byte swizzle for rows of 32 channels, 32-byte for 16): consecutive rows' 16-byte
// chunks fall in different shared-memory banks.
//
// Roles (320 threads, one persistent CTA per SM): warp 0 issues the tensor copies into a
// ring of slab stages; warp 1 allocates tensor memory and issues the MMAs (one elected
// thread), committing each stage back to the copier and each finished tile to the
// epilogue; two epilogue warpgroups (warps 2-5 and 6-9) take alternate tiles, each with its
// own accumulator buffer: they read the accumulators (tcgen05.ld, one TMEM lane quarter per
// warp), add the bias, apply ReLU and store BF16 rows (or, in the last layer, the FP32
// output of the real nodes). The epilogue is the longest role per tile, so two tiles of it
// run at once while the MMAs of a third proceed. Every wait is bounded: on expiry the CTA raises its abort flag and the error word,
// drains its copies and MMAs in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tt_net.h"

namespace ttgb {

namespace {

constexpr int kTileRows = 128;                 // M
constexpr int kTileStep = kTileRows - 2;       // output rows of one tile
#ifndef TTGB_TC_STAGES
#define TTGB_TC_STAGES 16
#endif
constexpr int kStages = TTGB_TC_STAGES;
constexpr int kThreads = 320;                  // copier, MMA, two epilogue warpgroups
// Two accumulator buffers of up to 3 x 32 columns.
constexpr int kBufCols = 128;
constexpr int kTmemCols = 256;

// KC: 8-channel chunks of an input row (2: C = 16, 4: C = 32); NO: output channels per dk
// (32, or 16 for the last layer).
template <int KC, int NO> struct Smem {
    static constexpr int ROW = KC * 16;                          // bytes of one row
    static constexpr int QW = 3 * NO * ROW;                      // weights of one (di, dj)
    static constexpr int W = 9 * QW;                             // [q][dk][co] rows, swizzled
    static constexpr int SLAB = kTileRows * ROW;
    static constexpr int A = (W + 1023) / 1024 * 1024;
    static constexpr int EXCH = A + kStages * SLAB;              // [2][4 quarters][2][2][32] float
    static constexpr int BAR = EXCH + 2 * 4 * 2 * 2 * 32 * 4;    // mbarriers
    static constexpr int NBAR = 2 * kStages + 5;                 // full, empty, acc x 4, drain
    static constexpr int MISC = BAR + NBAR * 8;                  // tmem address, abort flag
    static constexpr int TOTAL = MISC + 16 + 1024;               // + alignment slack
    // swizzle: 64 bytes for rows of 64 bytes, 32 for rows of 32 (descriptor layout code)
    static constexpr unsigned LAYOUT = ROW == 64 ? 4u : 6u;
    static constexpr unsigned SBO = 8 * ROW;                     // 8-row groups
};
static_assert(Smem<4, 32>::TOTAL <= 227 * 1024, "shared memory of one CTA");
static_assert(Smem<4, 32>::QW % 1024 == 0 && Smem<2, 32>::QW % 256 == 0 &&
                  Smem<4, 16>::QW % 512 == 0,
              "every weight block starts on a swizzle atom");

__device__ __forceinline__ unsigned saddr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(unsigned b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(unsigned b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bar_arrive(unsigned b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}

__device__ __forceinline__ bool bar_test(unsigned b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of the given parity. Returns false when the limit expired or
// another role of the CTA has aborted (then the caller stops).
__device__ __forceinline__ bool bar_wait(unsigned b, unsigned parity, unsigned long long limit,
                                         volatile int *abort) {
    unsigned long long t0 = 0;
    for (int spin = 0;; ++spin) {
        if (bar_test(b, parity)) return true;
        if ((spin & 63) == 63) {
            if (*abort) return false;
            const unsigned long long t = global_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit) {
                *abort = 1;
                return false;
            }
        }
    }
}

// Bounded wait used while tearing down (ignores the abort flag).
__device__ __forceinline__ void bar_drain(unsigned b, unsigned parity, unsigned long long limit) {
    const unsigned long long t0 = global_ns();
    while (!bar_test(b, parity) && global_ns() - t0 < limit) {
    }
}

// 128 rows of one grid starting at row `row` (may be negative or past the end: zero fill).
__device__ __forceinline__ void tma_rows(unsigned dst, const CUtensorMap *map, int row, int grid,
                                         unsigned b) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(0), "r"(row), "r"(grid), "r"(b)
        : "memory");
}

// Shared-memory matrix descriptor, K-major with swizzle `layout` (4: 64 B, 6: 32 B): rows of
// the swizzle width, 8-row groups sbo bytes apart; the leading offset is unused (encoded 1).
__device__ __forceinline__ unsigned long long mdesc(unsigned addr, unsigned sbo, unsigned layout) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | (1ull << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) |
           ((unsigned long long)layout << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N x M.
template <int N> __host__ __device__ constexpr unsigned idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
           ((unsigned)(kTileRows >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned d, unsigned long long a, unsigned long long b,
                                         unsigned id, unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b)
                 : "memory");
}

// 1 when c holds in every one of the 128 threads of epilogue group g (named barrier 1 + g).
__device__ __forceinline__ bool epi_all(int g, bool c) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %2, 0;\n bar.red.and.pred po, %1, 128, pi;\n"
        " selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"(1 + g), "r"((unsigned)c)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void epi_sync(int g) {
    asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Columns [taddr, +32), [+32, +64) and [+64, +96) of the thread's TMEM lane: three loads in
// flight and one wait, in one statement (the registers are only defined after the wait).
__device__ __forceinline__ void tmem_ld96(unsigned taddr, unsigned (&a)[32], unsigned (&b)[32],
                                          unsigned (&c)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%96];\n"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%97];\n"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%64, %65, %66, %67, %68, %69, %70, %71, %72, %73, %74, %75, %76, %77, %78, %79, %80, %81, %82, %83, %84, %85, %86, %87, %88, %89, %90, %91, %92, %93, %94, %95}, [%98];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
          "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]),
          "=r"(a[16]), "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]),
          "=r"(a[24]), "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]), "=r"(a[31]),
          "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]),
          "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15]),
          "=r"(b[16]), "=r"(b[17]), "=r"(b[18]), "=r"(b[19]), "=r"(b[20]), "=r"(b[21]), "=r"(b[22]), "=r"(b[23]),
          "=r"(b[24]), "=r"(b[25]), "=r"(b[26]), "=r"(b[27]), "=r"(b[28]), "=r"(b[29]), "=r"(b[30]), "=r"(b[31]),
          "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7]),
          "=r"(c[8]), "=r"(c[9]), "=r"(c[10]), "=r"(c[11]), "=r"(c[12]), "=r"(c[13]), "=r"(c[14]), "=r"(c[15]),
          "=r"(c[16]), "=r"(c[17]), "=r"(c[18]), "=r"(c[19]), "=r"(c[20]), "=r"(c[21]), "=r"(c[22]), "=r"(c[23]),
          "=r"(c[24]), "=r"(c[25]), "=r"(c[26]), "=r"(c[27]), "=r"(c[28]), "=r"(c[29]), "=r"(c[30]), "=r"(c[31])
        : "r"(taddr), "r"(taddr + 32), "r"(taddr + 64)
        : "memory");
}

__device__ __forceinline__ float tmem_ld1(unsigned taddr) {
    unsigned r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return __uint_as_float(r);
}

struct RowGeo {
    int nb, nr, nt, np;
    int Sj;             // n_p + 1
    int Si;             // (n_t + 1) Sj
    int R;              // rows of one grid: n_r Si
    int tiles;          // ceil(R / 126) per grid
};

__device__ __forceinline__ bool pad_row(const RowGeo &G, int n) {
    return n % G.Sj == G.np || (n / G.Sj) % (G.nt + 1) == G.nt;
}

// Epilogue modes: kEpiRelu writes ReLU(out + bias) as BF16 rows of 32 channels (a hidden
// layer); kEpiFinal writes channel 0 + bias as FP32 y[grid][node] (real nodes, the last
// layer); kEpiGate writes out * [gate > 0] as BF16 rows, gate being the BF16 rows of the
// layer below (training: the input gradient of a layer through the ReLU of the one below,
// computed with the flipped, transposed weights; no bias). Padding rows are written as zero.
constexpr int kEpiRelu = 0, kEpiFinal = 1, kEpiGate = 2;
template <int KC, int NO, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    conv3d_tc_kernel(const __grid_constant__ CUtensorMap map, RowGeo G,
                     const uint4 *__restrict__ wimg, const float *__restrict__ bias,
                     const uint4 *__restrict__ gate, void *__restrict__ out_, int *err,
                     unsigned long long limit) {
    constexpr bool FINAL = MODE == kEpiFinal;
    using L = Smem<KC, NO>;
    extern __shared__ unsigned char smem_raw[];
    const unsigned raw = saddr(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    unsigned char *sm = smem_raw + (base - raw);
    const unsigned sW = base, sA = base + L::A, sBar = base + L::BAR;
    unsigned *s_tmem = reinterpret_cast<unsigned *>(sm + L::MISC);
    volatile int *s_abort = reinterpret_cast<volatile int *>(sm + L::MISC + 4);
    auto full = [&](int s) { return sBar + 8u * s; };
    auto empty = [&](int s) { return sBar + 8u * (kStages + s); };
    auto acc_full = [&](int a) { return sBar + 8u * (2 * kStages + a); };
    auto acc_empty = [&](int a) { return sBar + 8u * (2 * kStages + 2 + a); };
    const unsigned drain = sBar + 8u * (2 * kStages + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // weights into shared memory (generic stores, made visible to the tensor cores below)
    for (int e = threadIdx.x; e < L::W / 16; e += kThreads)
        reinterpret_cast<uint4 *>(sm)[e] = wimg[e];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(full(s), 1);
            bar_init(empty(s), 1);
        }
        bar_init(acc_full(0), 1);
        bar_init(acc_full(1), 1);
        bar_init(acc_empty(0), 128);
        bar_init(acc_empty(1), 128);
        bar_init(drain, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *s_tmem;
    const long long total = (long long)G.nb * G.tiles;

    if (warp == 0) {
        if (lane == 0) {
            // copier: the nine slabs of every tile of this CTA, in order, into the stage ring
            int s = 0;
            unsigned ph = 0, armed = 0, armed_par = 0;
            bool ok = true;
            for (long long T = blockIdx.x; ok && T < total; T += gridDim.x) {
                const int g = (int)(T / G.tiles);
                const int n0 = (int)(T - (long long)g * G.tiles) * kTileStep;
                for (int q = 0; q < 9; ++q) {
                    if (!bar_wait(empty(s), ph ^ 1u, limit, s_abort)) { ok = false; break; }
                    bar_expect_tx(full(s), L::SLAB);
                    tma_rows(sA + s * L::SLAB, &map, n0 + (q / 3 - 1) * G.Si + (q % 3 - 1) * G.Sj - 1,
                             g, full(s));
                    armed |= 1u << s;
                    armed_par = (armed_par & ~(1u << s)) | (ph << s);
                    if (++s == kStages) { s = 0; ph ^= 1u; }
                }
            }
            // every copy issued has landed before the CTA may exit
            for (int q = 0; q < kStages; ++q)
                if (armed >> q & 1u) bar_drain(full(q), (armed_par >> q) & 1u, limit);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr unsigned ID = idesc_bf16<3 * NO>();
            int s = 0, a = 0;
            unsigned ph = 0, aph = 0;
            bool ok = true;
            for (long long T = blockIdx.x; ok && T < total; T += gridDim.x) {
                if (!bar_wait(acc_empty(a), aph ^ 1u, limit, s_abort)) break;
                tc_fence_after();
                const unsigned d = tmem + (unsigned)(a * kBufCols);
                for (int q = 0; q < 9; ++q) {
                    if (!bar_wait(full(s), ph, limit, s_abort)) { ok = false; break; }
                    const unsigned slab = sA + s * L::SLAB;
#pragma unroll
                    for (int h = 0; h < KC / 2; ++h) {
                        // K half h: 32 bytes into the swizzled rows; B: the (di, dj) weights of
                        // the three dk taps, rows [dk][co]
                        const unsigned long long ad = mdesc(slab + 32 * h, L::SBO, L::LAYOUT);
                        const unsigned long long bd = mdesc(sW + q * L::QW + 32 * h, L::SBO, L::LAYOUT);
                        mma_bf16(d, ad, bd, ID, (q | h) != 0);
                    }
                    mma_commit(empty(s));   // the stage is free once these MMAs have read it
                    if (++s == kStages) { s = 0; ph ^= 1u; }
                }
                if (!ok) break;
                mma_commit(acc_full(a));
                if (++a == 2) { a = 0; aph ^= 1u; }
            }
            // every MMA issued has completed before tensor memory is freed
            mma_commit(drain);
            bar_drain(drain, 0, limit);
        }
    } else {
        // epilogue group a (warps 2-5: a = 0, warps 6-9: a = 1) takes this CTA's tiles of
        // parity a, in accumulator buffer a; warp w reads TMEM lanes 32 (w % 4) ...
        const int a = (warp - 2) >> 2;
        const int quarter = warp & 3;
        const int m = quarter * 32 + lane;
        float *exch = reinterpret_cast<float *>(sm + L::EXCH);   // [2][4][2 lanes][2][32]
        float bz[FINAL ? 1 : 32];
#pragma unroll
        for (int c = 0; c < (FINAL ? 1 : 32); ++c) bz[c] = MODE == kEpiGate ? 0.0f : bias[c];
        unsigned aph = 0;
        for (long long T = blockIdx.x + (long long)a * gridDim.x; T < total; T += 2LL * gridDim.x) {
            // all 128 threads of the group agree (TMEM loads are warp-collective, the
            // exchange spans the group)
            if (!epi_all(a, bar_wait(acc_full(a), aph, limit, s_abort))) break;
            tc_fence_after();
            const unsigned taddr = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(a * kBufCols);
            float *ex = exch + a * 4 * 2 * 2 * 32;
            const int g = (int)(T / G.tiles);
            const int n = (int)(T - (long long)g * G.tiles) * kTileStep + m;
            const bool out_ok = m < kTileStep && n < G.R;
            if (FINAL) {
                const float d0 = tmem_ld1(taddr), d1 = tmem_ld1(taddr + NO),
                            d2 = tmem_ld1(taddr + 2 * NO);
                tc_fence_before();
                bar_arrive(acc_empty(a));
                if (lane < 2) {
                    ex[((quarter * 2 + lane) * 2 + 0) * 32] = d1;
                    ex[((quarter * 2 + lane) * 2 + 1) * 32] = d2;
                }
                epi_sync(a);
                float s1 = __shfl_down_sync(0xffffffffu, d1, 1);
                float s2 = __shfl_down_sync(0xffffffffu, d2, 2);
                if (quarter < 3) {
                    if (lane == 31) s1 = ex[(((quarter + 1) * 2 + 0) * 2 + 0) * 32];
                    if (lane >= 30) s2 = ex[(((quarter + 1) * 2 + lane - 30) * 2 + 1) * 32];
                }
                if (out_ok && !pad_row(G, n)) {
                    const int k = n % G.Sj, j = (n / G.Sj) % (G.nt + 1), i = n / G.Si;
                    const long long node = ((long long)i * G.nt + j) * G.np + k;
                    reinterpret_cast<float *>(out_)[(long long)g * G.nr * G.nt * G.np + node] =
                        (d0 + s1) + s2 + bz[0];
                }
            } else {
                float d0[32], d1[32], d2[32];
                {
                    unsigned r0[32], r1[32], r2[32];
                    tmem_ld96(taddr, r0, r1, r2);
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        d0[c] = __uint_as_float(r0[c]);
                        d1[c] = __uint_as_float(r1[c]);
                        d2[c] = __uint_as_float(r2[c]);
                    }
                }
                tc_fence_before();
                bar_arrive(acc_empty(a));
                if (lane < 2) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        ex[((quarter * 2 + lane) * 2 + 0) * 32 + c] = d1[c];
                        ex[((quarter * 2 + lane) * 2 + 1) * 32 + c] = d2[c];
                    }
                }
                epi_sync(a);
                const bool zero = !out_ok || pad_row(G, n);
                unsigned gw[16];   // kEpiGate: the gate row's 32 BF16 channels
                if (MODE == kEpiGate && !zero) {
                    const uint4 *gr = gate + ((long long)g * G.R + n) * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint4 v = gr[c];
                        gw[4 * c] = v.x;
                        gw[4 * c + 1] = v.y;
                        gw[4 * c + 2] = v.z;
                        gw[4 * c + 3] = v.w;
                    }
                }
                unsigned w[16];
#pragma unroll
                for (int c = 0; c < 32; c += 2) {
                    float v[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        float s1 = __shfl_down_sync(0xffffffffu, d1[c + u], 1);
                        float s2 = __shfl_down_sync(0xffffffffu, d2[c + u], 2);
                        if (quarter < 3) {
                            if (lane == 31) s1 = ex[(((quarter + 1) * 2 + 0) * 2 + 0) * 32 + c + u];
                            if (lane >= 30) s2 = ex[(((quarter + 1) * 2 + lane - 30) * 2 + 1) * 32 + c + u];
                        }
                        if (MODE == kEpiGate) {
                            const unsigned short hb = (unsigned short)(gw[c / 2] >> (16 * u));
                            const bool open = !zero && __bfloat162float(__ushort_as_bfloat16(hb)) > 0.0f;
                            v[u] = open ? (d0[c + u] + s1) + s2 : 0.0f;
                        } else {
                            v[u] = zero ? 0.0f : fmaxf((d0[c + u] + s1) + s2 + bz[c + u], 0.0f);
                        }
                    }
                    const __nv_bfloat162 p = __floats2bfloat162_rn(v[0], v[1]);
                    w[c / 2] = *reinterpret_cast<const unsigned *>(&p);
                }
                if (out_ok) {
                    uint4 *o = reinterpret_cast<uint4 *>(out_) + ((long long)g * G.R + n) * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        o[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
                }
            }
            aph ^= 1u;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
    if (threadIdx.x == 0 && *s_abort) atomicExch(err, 1);
}

// Features [grid][node][6] (FP32) -> input rows [grid][R][16] (BF16; channels 6-15 and the
// padding rows zero).
__global__ void pack_features_kernel(RowGeo G, const float *__restrict__ x, uint4 *__restrict__ xp) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)G.nb * G.R) return;
    const int g = (int)(q / G.R), n = (int)(q - (long long)g * G.R);
    unsigned w[4] = {0u, 0u, 0u, 0u};
    if (!pad_row(G, n)) {
        const int k = n % G.Sj, j = (n / G.Sj) % (G.nt + 1), i = n / G.Si;
        const float *f = x + ((long long)g * G.nr * G.nt * G.np + ((long long)i * G.nt + j) * G.np + k) *
                                 kNetFeatures;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const __nv_bfloat162 p = __floats2bfloat162_rn(f[2 * c], f[2 * c + 1]);
            w[c] = *reinterpret_cast<const unsigned *>(&p);
        }
    }
    xp[2 * q] = make_uint4(w[0], w[1], w[2], w[3]);
    xp[2 * q + 1] = make_uint4(0u, 0u, 0u, 0u);
}

// dL/dy [grid][node] (FP32) -> rows [grid][R][16] (BF16, channel 0; the rest and the padding
// rows zero): the input of the last layer's transposed convolution in training.
__global__ void pack_dy_kernel(RowGeo G, const float *__restrict__ dy, uint4 *__restrict__ out) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)G.nb * G.R) return;
    const int g = (int)(q / G.R), n = (int)(q - (long long)g * G.R);
    unsigned w0 = 0u;
    if (!pad_row(G, n)) {
        const int k = n % G.Sj, j = (n / G.Sj) % (G.nt + 1), i = n / G.Si;
        const float v = dy[(long long)g * G.nr * G.nt * G.np + ((long long)i * G.nt + j) * G.np + k];
        const __nv_bfloat162 p = __floats2bfloat162_rn(v, 0.0f);
        w0 = *reinterpret_cast<const unsigned *>(&p);
    }
    out[2 * q] = make_uint4(w0, 0u, 0u, 0u);
    out[2 * q + 1] = make_uint4(0u, 0u, 0u, 0u);
}

// Layer l's weights W[27][cin][cout] (FP32) -> the shared-memory image of the B operands
// (BF16): for q = (di, dj), rows (dk, co) of C = 8 KC input channels (tap t = 3 q + dk; zero
// beyond cin and cout), each row's 16-byte chunks placed as the tensor cores' swizzle of the
// row width expects them (chunk c of row r at c ^ ((r >> 1) & 3) for 64-byte rows,
// c ^ ((r >> 2) & 1) for 32-byte rows).
__global__ void weight_image_kernel(const float *__restrict__ w, int cin, int cout, int KC, int NO,
                                    __nv_bfloat16 *__restrict__ img) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // logical element (q, dk, co, ci)
    if (e >= 27 * NO * KC * 8) return;
    const int C = 8 * KC;
    const int ci = e % C, co = (e / C) % NO, dk = (e / (C * NO)) % 3, q = e / (3 * C * NO);
    const int t = 3 * q + dk;
    const float v = ci < cin && co < cout ? w[((size_t)t * cin + ci) * cout + co] : 0.0f;
    const int r = dk * NO + co;                     // row within the (di, dj) block
    const int c = ci / 8;
    const int cs = KC == 4 ? c ^ ((r >> 1) & 3) : c ^ ((r >> 2) & 1);
    img[((size_t)q * 3 * NO + r) * C + cs * 8 + ci % 8] = __float2bfloat16_rn(v);
}

// ------------------------------------------------------------------------ weight gradients
//
// Training: the weight gradient of a layer with input rows X (C_in BF16 channels) and
// output-gradient rows G (C_g channels),
//   dW[t][ci][co] = sum_r X[r + s(di, dj) + dk - 1][ci] G[r][co],   t = 9 di + 3 dj + dk,
// with s(di, dj) = (di - 1) Si + (dj - 1) Sj the row shift of the (di, dj) taps. Writing
// r' = r + dk - 1 moves the dk shift onto G: dW[t] = sum_r' X[r' + s(di, dj)] G[r' - dk + 1],
// r' over [-1, R + 1) (rows outside [0, R) are zero). A chunk of 64 rows r' is one GEMM step
// with K = rows: A = the nine (di, dj) slabs of X rows, B = the three dk slabs of G rows. Both
// are the row buffers as they are (channels contiguous), i.e. MN-major operands: an M group
// of 128 stacks 128 / C_in slabs (one swizzle atom of C_in channels each, LBO apart), N = 3
// C_g stacks the three dk slabs the same way, and 8-row groups are SBO apart. The
// accumulator of an M group holds, in TMEM lane (slab, ci) and column (dk, co), the sums of
// its taps over this CTA's chunks. One slab position of the last M
// group holds ones: its lanes collect sum_r G[r][co], the bias gradient (dk = 1 reads every
// row of G once). Each CTA writes its sums as a partial row; wgrad_reduce sums the rows in a
// fixed order, so the result is bitwise reproducible. Roles: warp 0 issues the tensor copies
// into a ring of stages, warp 1 owns the tensor memory and issues the MMAs, warps 2-5 read
// the accumulators once at the end. Every wait is bounded as in conv3d_tc_kernel.
constexpr int kWgRows = 64;        // K rows of one chunk
constexpr int kWgStages = 3;
constexpr int kWgThreads = 192;
constexpr int kWgTmemCols = 512;

template <int KCI, int KCG> struct WgSmem {
    static constexpr int CI = KCI * 8, CG = KCG * 8;             // channels of X and G rows
    static constexpr int XROW = KCI * 16, GROW = KCG * 16;        // bytes of one row
    static constexpr int SPG = 128 / CI;                          // slabs of one M group
    static constexpr int MG = (9 + 1 + SPG - 1) / SPG;            // M groups: 9 slabs + ones
    static constexpr int ONES = MG * SPG - 1;                     // slab position of the ones
    static constexpr int XSLAB = kWgRows * XROW, GSLAB = kWgRows * GROW;
    static constexpr int GOFF = MG * SPG * XSLAB;                 // G slabs within a stage
    static constexpr int STAGE = GOFF + 3 * GSLAB;
    static constexpr int BAR = kWgStages * STAGE;
    static constexpr int NBAR = 2 * kWgStages + 2;                // full, empty, acc, drain
    static constexpr int MISC = BAR + NBAR * 8;
    static constexpr int TOTAL = MISC + 16 + 1024;
    static constexpr unsigned XLAYOUT = XROW == 64 ? 4u : 6u, GLAYOUT = GROW == 64 ? 4u : 6u;
    static constexpr int N = 3 * CG;   // one MMA covers the three dk slabs (N atoms LBO apart)
};
static_assert(WgSmem<4, 4>::TOTAL <= 227 * 1024 && WgSmem<4, 4>::STAGE % 1024 == 0 &&
                  WgSmem<4, 2>::STAGE % 1024 == 0 && WgSmem<2, 4>::STAGE % 1024 == 0,
              "weight-gradient stages: shared memory and swizzle-atom alignment");
static_assert(WgSmem<4, 4>::MG * WgSmem<4, 4>::N <= kWgTmemCols &&
                  WgSmem<2, 4>::MG * WgSmem<2, 4>::N <= kWgTmemCols,
              "weight-gradient accumulators fit the tensor memory");

// Shared-memory matrix descriptor of an MN-major operand with swizzle `layout`: swizzle atoms
// of the MN dimension lbo bytes apart, 8-row groups of the K dimension sbo bytes apart.
__device__ __forceinline__ unsigned long long mdesc_mn(unsigned addr, unsigned lbo, unsigned sbo,
                                                       unsigned layout) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) |
           ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) |
           ((unsigned long long)layout << 61);
}

// Instruction descriptor of kind::f16 with both operands MN-major (FP32 accumulator, BF16).
template <int N> __host__ __device__ constexpr unsigned idesc_bf16_mn() {
    return idesc_bf16<N>() | (1u << 15) | (1u << 16);
}

template <int N> __device__ __forceinline__ void tmem_ld_cols(unsigned taddr, float (&v)[N]);
template <> __device__ __forceinline__ void tmem_ld_cols<16>(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}
template <> __device__ __forceinline__ void tmem_ld_cols<32>(unsigned taddr, float (&v)[32]) {
    float a[16], b[16];
    tmem_ld_cols<16>(taddr, a);
    tmem_ld_cols<16>(taddr + 16, b);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        v[c] = a[c];
        v[16 + c] = b[c];
    }
}

template <int KCI, int KCG>
__global__ void __launch_bounds__(kWgThreads, 1)
    conv3d_wgrad_tc_kernel(const __grid_constant__ CUtensorMap mx,
                           const __grid_constant__ CUtensorMap mgr, RowGeo G, int cin, int cout,
                           float *__restrict__ partial, int *err, unsigned long long limit) {
    using L = WgSmem<KCI, KCG>;
    extern __shared__ unsigned char smem_raw[];
    const unsigned raw = saddr(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    unsigned char *sm = smem_raw + (base - raw);
    const unsigned sBar = base + L::BAR;
    unsigned *s_tmem = reinterpret_cast<unsigned *>(sm + L::MISC);
    volatile int *s_abort = reinterpret_cast<volatile int *>(sm + L::MISC + 4);
    auto full = [&](int s) { return sBar + 8u * s; };
    auto empty = [&](int s) { return sBar + 8u * (kWgStages + s); };
    const unsigned acc_full = sBar + 8u * (2 * kWgStages), drain = acc_full + 8u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long cpg = (G.R + 2 + kWgRows - 1) / kWgRows;   // chunks of one grid
    const long long total = (long long)G.nb * cpg;

    // the ones slab of every stage (never overwritten by the copies)
    for (int s = 0; s < kWgStages; ++s) {
        uint4 *o = reinterpret_cast<uint4 *>(sm + s * L::STAGE + L::ONES * L::XSLAB);
        for (int e = threadIdx.x; e < L::XSLAB / 16; e += kWgThreads)
            o[e] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);  // BF16 1.0
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            bar_init(full(s), 1);
            bar_init(empty(s), 1);
        }
        bar_init(acc_full, 1);
        bar_init(drain, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(s_tmem)),
                     "r"(kWgTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            // copier: per chunk, nine X slabs and three G slabs into one stage
            int s = 0;
            unsigned ph = 0, armed = 0, armed_par = 0;
            for (long long c = blockIdx.x; c < total; c += gridDim.x) {
                const int g = (int)(c / cpg);
                const int r0 = (int)(c - (long long)g * cpg) * kWgRows - 1;
                if (!bar_wait(empty(s), ph ^ 1u, limit, s_abort)) break;
                bar_expect_tx(full(s), 9 * L::XSLAB + 3 * L::GSLAB);
                const unsigned st = base + s * L::STAGE;
                for (int q = 0; q < 9; ++q)
                    tma_rows(st + q * L::XSLAB, &mx, r0 + (q / 3 - 1) * G.Si + (q % 3 - 1) * G.Sj,
                             g, full(s));
                for (int dk = 0; dk < 3; ++dk)
                    tma_rows(st + L::GOFF + dk * L::GSLAB, &mgr, r0 - dk + 1, g, full(s));
                armed |= 1u << s;
                armed_par = (armed_par & ~(1u << s)) | (ph << s);
                if (++s == kWgStages) { s = 0; ph ^= 1u; }
            }
            for (int q = 0; q < kWgStages; ++q)
                if (armed >> q & 1u) bar_drain(full(q), (armed_par >> q) & 1u, limit);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr unsigned ID = idesc_bf16_mn<L::N>();
            int s = 0;
            unsigned ph = 0;
            bool ok = true, first = true;
            for (long long c = blockIdx.x; c < total; c += gridDim.x) {
                if (!bar_wait(full(s), ph, limit, s_abort)) { ok = false; break; }
                tc_fence_after();
                const unsigned st = base + s * L::STAGE;
                for (int mg = 0; mg < L::MG; ++mg)
#pragma unroll
                    for (int ks = 0; ks < kWgRows / 16; ++ks) {
                        // A: the M group's slabs; B: the three dk slabs, one N atom each
                        const unsigned long long ad =
                            mdesc_mn(st + mg * L::SPG * L::XSLAB + ks * 16 * L::XROW, L::XSLAB,
                                     8 * L::XROW, L::XLAYOUT);
                        const unsigned long long bd =
                            mdesc_mn(st + L::GOFF + ks * 16 * L::GROW, L::GSLAB, 8 * L::GROW,
                                     L::GLAYOUT);
                        mma_bf16(tmem + (unsigned)(mg * L::N), ad, bd, ID, !(first && ks == 0));
                    }
                mma_commit(empty(s));   // the stage is free once these MMAs have read it
                first = false;
                if (++s == kWgStages) { s = 0; ph ^= 1u; }
            }
            if (ok) mma_commit(acc_full);
            mma_commit(drain);
            bar_drain(drain, 0, limit);
        }
    } else {
        // warps 2-5: TMEM lane quarter warp % 4; lane m = (slab within the M group, channel)
        const int quarter = warp & 3;
        const int m = quarter * 32 + lane;
        const int p_in = m / L::CI, ch = m - p_in * L::CI;
        if (epi_all(0, bar_wait(acc_full, 0, limit, s_abort))) {
            tc_fence_after();
            for (int dk = 0; dk < 3; ++dk)
                for (int mg = 0; mg < L::MG; ++mg) {
                    float v[L::CG];
                    tmem_ld_cols<L::CG>(tmem + ((unsigned)(quarter * 32) << 16) +
                                            (unsigned)(mg * L::N + dk * L::CG),
                                        v);
                    const int p = mg * L::SPG + p_in;
                    float *row = nullptr;
                    if (p < 9 && ch < cin)
                        row = partial + ((size_t)blockIdx.x * 28 + 3 * p + dk) * 1024 + ch * cout;
                    else if (p == L::ONES && ch == 0 && dk == 1)
                        row = partial + ((size_t)blockIdx.x * 28 + 27) * 1024;
                    if (row)
#pragma unroll
                        for (int n = 0; n < L::CG; ++n)
                            if (n < cout) row[n] = v[n];
                }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kWgTmemCols)
                     : "memory");
    }
    if (threadIdx.x == 0 && *s_abort) atomicExch(err, 1);
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

PFN_cuTensorMapEncodeTiled_v12000 map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor map over rows of 8 KC BF16 channels: dims (channels, R rows, nb grids); a box is
// box_rows rows of one grid, swizzled as the descriptors expect.
cudaError_t encode_rows(CUtensorMap *map, const void *base, const RowGeo &G, int KC,
                        int box_rows = kTileRows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t row = (cuuint64_t)KC * 16;
    cuuint64_t dims[3] = {(cuuint64_t)KC * 8, (cuuint64_t)G.R, (cuuint64_t)G.nb};
    cuuint64_t strides[2] = {row, row * (cuuint64_t)G.R};
    cuuint32_t box[3] = {(cuuint32_t)KC * 8, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           KC == 4 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int KC, int NO, int MODE>
cudaError_t launch_layer(const void *in, const RowGeo &G, const __nv_bfloat16 *wimg,
                         const float *bias, void *out, int n_sm, int *err,
                         unsigned long long limit, cudaStream_t st, const void *gate = nullptr) {
    CUtensorMap map;
    cudaError_t e = encode_rows(&map, in, G, KC);
    if (e != cudaSuccess) return e;
    // more than half the shared memory of an SM: one CTA per SM, which owns its TMEM
    constexpr int smem = Smem<KC, NO>::TOTAL > 120 * 1024 ? Smem<KC, NO>::TOTAL : 120 * 1024;
    const void *fn = (const void *)conv3d_tc_kernel<KC, NO, MODE>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const long long total = (long long)G.nb * G.tiles;
    const unsigned grid = (unsigned)(total < n_sm ? total : n_sm);
    conv3d_tc_kernel<KC, NO, MODE><<<grid, kThreads, smem, st>>>(
        map, G, reinterpret_cast<const uint4 *>(wimg), bias, reinterpret_cast<const uint4 *>(gate),
        out, err, limit);
    return cudaGetLastError();
}

// Weight and bias gradients of one layer on the tensor cores: per-CTA partial rows, then the
// fixed-order reduction into gw [27][cin][cout] and gb [cout].
template <int KCI, int KCG>
cudaError_t launch_wgrad(const void *in, const void *g, const RowGeo &G, int cin, int cout,
                         float *partial, float *gw, float *gb, int n_sm, int *err,
                         unsigned long long limit, cudaStream_t st) {
    using L = WgSmem<KCI, KCG>;
    if (cin > L::CI || cout > L::CG || cin * cout > 1024) return cudaErrorInvalidValue;
    CUtensorMap mx, mgr;
    cudaError_t e = encode_rows(&mx, in, G, KCI, kWgRows);
    if (e != cudaSuccess) return e;
    if ((e = encode_rows(&mgr, g, G, KCG, kWgRows)) != cudaSuccess) return e;
    // more than half the shared memory of an SM: one CTA per SM, which owns its TMEM
    constexpr int smem = L::TOTAL > 120 * 1024 ? L::TOTAL : 120 * 1024;
    const void *fn = (const void *)conv3d_wgrad_tc_kernel<KCI, KCG>;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
        return e;
    const long long total = (long long)G.nb * ((G.R + 2 + kWgRows - 1) / kWgRows);
    long long grid = n_sm < kWgradBlocks ? n_sm : kWgradBlocks;
    if (grid > total) grid = total;
    conv3d_wgrad_tc_kernel<KCI, KCG><<<(unsigned)grid, kWgThreads, smem, st>>>(
        mx, mgr, G, cin, cout, partial, err, limit);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return run_wgrad_reduce(cin, cout, (int)grid, partial, gw, gb, st);
}

RowGeo row_geo(const ConvDims &d) {
    RowGeo G;
    G.nb = d.nb;
    G.nr = d.D;
    G.nt = d.H;
    G.np = d.W;
    G.Sj = d.W + 1;
    G.Si = (d.H + 1) * G.Sj;
    G.R = d.D * G.Si;
    G.tiles = (G.R + kTileStep - 1) / kTileStep;
    return G;
}

}  // namespace

size_t net_rows(const ConvDims &d) { return (size_t)row_geo(d).R; }

size_t net_weight_image_elems() {
    return (size_t)27 * 8 * (2 * 32 + 4 * 32 + 4 * 32 + 4 * 16);
}

// Offsets of the four layers' images in the concatenated weight image.
static size_t image_offset(int l) {
    const size_t sz[kNetLayers] = {27u * 2 * 32 * 8, 27u * 4 * 32 * 8, 27u * 4 * 32 * 8,
                                   27u * 4 * 16 * 8};
    size_t o = 0;
    for (int q = 0; q < l; ++q) o += sz[q];
    return o;
}

cudaError_t run_net_weight_images(const float *theta, __nv_bfloat16 *img, cudaStream_t st) {
    const int KC[kNetLayers] = {2, 4, 4, 4}, NO[kNetLayers] = {32, 32, 32, 16};
    for (int l = 0; l < kNetLayers; ++l) {
        const int n = 27 * KC[l] * NO[l] * 8;
        weight_image_kernel<<<blocks_for(n, 256), 256, 0, st>>>(
            theta + net_weight_offset(l), kNetCin[l], kNetCout[l], KC[l], NO[l], img + image_offset(l));
    }
    return cudaGetLastError();
}

// Sizes of the transposed layers' images (layers 1-3; layer 0 has none): the gradient of
// layer l's output (cout_l channels, 1 -> 16 padded for the last layer) to its input (32).
static size_t image_offset_t(int l) {
    const size_t sz[kNetLayers] = {0u, 27u * 4 * 32 * 8, 27u * 4 * 32 * 8, 27u * 2 * 32 * 8};
    size_t o = 0;
    for (int q = 0; q < l; ++q) o += sz[q];
    return o;
}
size_t net_tweight_image_elems() { return image_offset_t(kNetLayers - 1) + 27u * 2 * 32 * 8; }

size_t net_train_row_elems(const ConvDims &d) {
    return (size_t)row_geo(d).R * d.nb * (16 + 3 * 32 + 16 + 3 * 32);
}

cudaError_t run_net_loss_grad_tc(const ConvDims &d, const float *theta, const float *x,
                                 const float *target, const float *mask, float *grad,
                                 double *loss, __nv_bfloat16 *img, __nv_bfloat16 *timg,
                                 float *wt, __nv_bfloat16 *rows, float *y, float *dy,
                                 float *partial, double *scratch, int n_sm, int *err,
                                 unsigned long long limit, cudaStream_t st) {
    const RowGeo G = row_geo(d);
    const size_t R = (size_t)G.R * G.nb;
    // rows: X (16 channels), A1..A3 (32), DY (16), G3, G2, G1 (32); A_l is layer l's output
    __nv_bfloat16 *X = rows, *A[3], *DY, *Gr[3];
    A[0] = X + 16 * R;
    A[1] = A[0] + 32 * R;
    A[2] = A[1] + 32 * R;
    DY = A[2] + 32 * R;
    Gr[0] = DY + 16 * R;      // gradient at the output of layer 1 (before its ReLU)
    Gr[1] = Gr[0] + 32 * R;   // ... of layer 2
    Gr[2] = Gr[1] + 32 * R;   // ... of layer 3
    cudaError_t e = run_net_weight_images(theta, img, st);
    if (e != cudaSuccess) return e;
    for (int l = 1; l < kNetLayers; ++l) {
        const int ci = kNetCin[l], co = kNetCout[l];
        if ((e = run_conv3d_flip(ci, co, theta + net_weight_offset(l), wt, st)) != cudaSuccess)
            return e;
        const int KC = co <= 16 ? 2 : 4, n = 27 * KC * 32 * 8;
        weight_image_kernel<<<blocks_for(n, 256), 256, 0, st>>>(wt, co, ci, KC, 32,
                                                                timg + image_offset_t(l));
    }
    pack_features_kernel<<<blocks_for((long long)R, 256), 256, 0, st>>>(
        G, x, reinterpret_cast<uint4 *>(X));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const float *bias[kNetLayers];
    for (int l = 0; l < kNetLayers; ++l)
        bias[l] = theta + net_weight_offset(l) + 27 * kNetCin[l] * kNetCout[l];
    // forward, every layer's output kept
    if ((e = launch_layer<2, 32, kEpiRelu>(X, G, img + image_offset(0), bias[0], A[0], n_sm, err,
                                           limit, st)) != cudaSuccess)
        return e;
    for (int l = 1; l < 3; ++l)
        if ((e = launch_layer<4, 32, kEpiRelu>(A[l - 1], G, img + image_offset(l), bias[l], A[l],
                                               n_sm, err, limit, st)) != cudaSuccess)
            return e;
    if ((e = launch_layer<4, 16, kEpiFinal>(A[2], G, img + image_offset(3), bias[3], y, n_sm, err,
                                            limit, st)) != cudaSuccess)
        return e;
    if ((e = run_mse((long long)d.nb * d.D * d.H * d.W, y, target, mask, dy, scratch, loss, st)) !=
        cudaSuccess)
        return e;
    pack_dy_kernel<<<blocks_for((long long)R, 256), 256, 0, st>>>(G, dy, reinterpret_cast<uint4 *>(DY));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // backward, last layer first: the weight gradient of layer l from its input rows and the
    // gradient rows of its output (conv3d_wgrad_tc_kernel); the gradient of its input through
    // the transposed convolution, gated by the ReLU of the layer below
    const __nv_bfloat16 *gout = DY;
    int gch = 16;
    for (int l = kNetLayers - 1; l >= 0; --l) {
        const int ci = kNetCin[l], co = kNetCout[l];
        const __nv_bfloat16 *in = l == 0 ? X : A[l - 1];
        float *gw = grad + net_weight_offset(l);
        e = l == 0 ? launch_wgrad<2, 4>(in, gout, G, ci, co, partial, gw, gw + 27 * ci * co, n_sm,
                                        err, limit, st)
            : gch == 16 ? launch_wgrad<4, 2>(in, gout, G, ci, co, partial, gw, gw + 27 * ci * co,
                                             n_sm, err, limit, st)
                        : launch_wgrad<4, 4>(in, gout, G, ci, co, partial, gw, gw + 27 * ci * co,
                                             n_sm, err, limit, st);
        if (e != cudaSuccess) return e;
        if (l == 0) break;
        __nv_bfloat16 *gin = Gr[l - 1];
        e = l == kNetLayers - 1
                ? launch_layer<2, 32, kEpiGate>(gout, G, timg + image_offset_t(l), nullptr, gin,
                                                n_sm, err, limit, st, A[l - 1])
                : launch_layer<4, 32, kEpiGate>(gout, G, timg + image_offset_t(l), nullptr, gin,
                                                n_sm, err, limit, st, A[l - 1]);
        if (e != cudaSuccess) return e;
        gout = gin;
        gch = 32;
    }
    return cudaGetLastError();
}

cudaError_t run_net_infer(const ConvDims &d, const float *theta, const __nv_bfloat16 *img,
                          const float *x, __nv_bfloat16 *a, __nv_bfloat16 *b, float *y, int n_sm,
                          int *err, unsigned long long limit, cudaStream_t st) {
    static_assert(kNetHidden == 32 && kNetFeatures <= 16 && kNetCout[3] <= 16,
                  "layer shapes of the tensor-core kernels");
    const RowGeo G = row_geo(d);
    // the input rows live in b until layer 2 overwrites it
    pack_features_kernel<<<blocks_for((long long)G.nb * G.R, 256), 256, 0, st>>>(
        G, x, reinterpret_cast<uint4 *>(b));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float *bias[kNetLayers];
    for (int l = 0; l < kNetLayers; ++l)
        bias[l] = theta + net_weight_offset(l) + 27 * kNetCin[l] * kNetCout[l];
    if ((e = launch_layer<2, 32, kEpiRelu>(b, G, img + image_offset(0), bias[0], a, n_sm, err, limit, st)) !=
        cudaSuccess)
        return e;
    if ((e = launch_layer<4, 32, kEpiRelu>(a, G, img + image_offset(1), bias[1], b, n_sm, err, limit, st)) !=
        cudaSuccess)
        return e;
    if ((e = launch_layer<4, 32, kEpiRelu>(b, G, img + image_offset(2), bias[2], a, n_sm, err, limit, st)) !=
        cudaSuccess)
        return e;
    return launch_layer<4, 16, kEpiFinal>(a, G, img + image_offset(3), bias[3], y, n_sm, err, limit, st);
}

}  // namespace ttgb
