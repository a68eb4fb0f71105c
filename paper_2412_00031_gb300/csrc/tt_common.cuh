// Device-side building blocks shared by the CUDA kernels of libttgb: grid constants, the
// per-source factor T0 (Sec. 3.1), the per-node model record and a bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ttgb {

// Empty slot in integer index maps. A byte pattern, so that cudaMemset(p, 0x7f, n) fills a
// map with it; larger than any index the library builds.
constexpr int kNone = 0x7f7f7f7f;

// Status word written by kernels (0 = ok). Values mirror tt_status.
enum DevStatus : int { kDevOk = 0, kDevTimeout = 4, kDevBadIndex = 1 };

// Uniform grid (r ascending from r0, theta = latitude, phi = longitude), Sec. 2.1.
struct GridC {
    int nr, nt, np;
    int flat;
    long long N;
    double r0, dr, t0, dt, p0, dp, re;
};

__host__ __device__ inline long long node_index(const GridC &g, int i, int j, int k) {
    return ((long long)i * g.nt + j) * g.np + k;
}

// Per-source constants of the multiplicative factor T0 = s0 sqrt(D^T M0^-1 D), D the offset
// to the source in the source's local (up, north, east) frame, M0 = M(xi0, eta0) of Eq. "4".
// Built once per call in FP64 by the source set-up kernel.
struct SrcC {
    double fr, ft, fp;     // fractional grid index of the source
    double frr;            // fr - ir, so that i - fr = (i - ir) - frr without cancellation
    double s0, inv_s0;
    double b11, b12, b22;  // theta-phi block of M0^-1 (the r-r entry is 1)
    double sts, cts;       // sin, cos of the source latitude
    int ir;                // floor(fr)
    int ci, cj, ck;        // node nearest the source: centre of the 3x3x3 fixed set
};

// Per-node model record of the forward sweep (shared by all sources of a batch):
// s, xi, eta, and the Lax-Friedrichs coefficients c_t = sqrt(1-2xi) e_t,
// c_p = sqrt(1+2xi) e_p, invW = 1 / (2 (e_r + c_t + c_p)), with e_d = 1 / (2 delta_d h_d).
template <typename F> struct alignas(sizeof(F) * 8) NodeRec {
    F s, xi, eta, ct, cp, invW, et, ep;
};

template <typename F> struct Vec2 { F x, y; };
template <typename F> struct alignas(sizeof(F) * 4) Vec4 { F x, y, z, w; };

__device__ __forceinline__ bool in_fixed_set(int ci, int cj, int ck, int i, int j, int k) {
    return abs(i - ci) <= 1 && abs(j - cj) <= 1 && abs(k - ck) <= 1;
}

// Per-source values held in registers by the sweep kernels.
template <typename F> struct SrcReg {
    F frr, dr, s0, inv_s0, b11, b12, b22, sts, cts;
    int ir, ci, cj, ck;
};

template <typename F> __device__ __forceinline__ SrcReg<F> load_src(const SrcC *S, int b, double dr) {
    SrcReg<F> r;
    const SrcC &c = S[b];
    r.frr = (F)c.frr; r.ir = c.ir; r.dr = (F)dr; r.s0 = (F)c.s0; r.inv_s0 = (F)c.inv_s0;
    r.b11 = (F)c.b11; r.b12 = (F)c.b12; r.b22 = (F)c.b22;
    r.sts = (F)c.sts; r.cts = (F)c.cts;
    r.ci = c.ci; r.cj = c.cj; r.ck = c.ck;
    return r;
}

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
#ifndef TTGB_SQRT_APPROX
#define TTGB_SQRT_APPROX 1
#endif
// FP32: the hardware square root (sqrt.approx.f32), a single deterministic instruction.
#if TTGB_SQRT_APPROX
__device__ __forceinline__ float sqrt_(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
#else
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
#endif
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }

// Rounding-explicit arithmetic: each call is one IEEE operation that the compiler neither
// contracts nor reorders, so every kernel that calls lf_core performs bit-identical
// arithmetic whatever code surrounds it.
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float div_(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_(double a, double b) { return __ddiv_rn(a, b); }

// Offset D = (up, north, east) of node (i, r, theta) from the source in the source's frame.
// Rounding-explicit (like every function below), so the factor is the same bits in every
// kernel that computes it.
template <typename F>
__device__ __forceinline__ void source_offset(const SrcReg<F> &S, int i, F r, F cth, Vec2<F> tT,
                                              Vec2<F> tP, bool flat, F &du, F &dn, F &de) {
    du = mul_(sub_((F)(i - S.ir), S.frr), S.dr);
    if (flat) {
        dn = tT.x;
        de = tP.x;
    } else {
        du = sub_(du, mul_(r, fma_(mul_(S.cts, cth), tP.y, tT.y)));
        dn = mul_(r, fma_(mul_(S.sts, cth), tP.y, tT.x));
        de = mul_(mul_(r, cth), tP.x);
    }
}

// T0 at node (i, j, k) for one source, returned as 1/T0 and u = p0 / T0, where p0 is the
// gradient of T0 in the node's physical components (d_r, d_theta / r, d_phi / (r cos theta)).
// Spherical geometry: with dth = theta - theta_s and dph = phi - phi_s,
//   D_up    = (r - r_s) - r [(1 - cos dth) + cos th_s cos th (1 - cos dph)]
//   D_north = r [sin dth + sin th_s cos th (1 - cos dph)]
//   D_east  = r cos th sin dph
// (no cancellation: the small angle terms come from tables built in FP64), and p0 is the
// source-frame gradient s0^2 M0^-1 D / T0 rotated into the node frame by Q_ab = e_a . E_b.
// tabT = (sin dth, 1 - cos dth) at the node's latitude, tabP = (sin dph, 1 - cos dph).
// Flat geometry: tabT = (R_E dth, 0), tabP = (R_E dph, 0), D = (r - r_s, tabT.x, tabP.x), Q = I.
template <typename F>
__device__ __forceinline__ F factor_T0(const SrcReg<F> &S, int i, F r, F cth, F sth,
                                       Vec2<F> tT, Vec2<F> tP, bool flat, F &ur, F &ut, F &up) {
    F du, dn, de;
    source_offset<F>(S, i, r, cth, tT, tP, flat, du, dn, de);
    const F wn = fma_(S.b11, dn, mul_(S.b12, de));
    const F we = fma_(S.b12, dn, mul_(S.b22, de));
    const F q = fma_(du, du, fma_(dn, wn, mul_(de, we)));
    const F rho = rsqrt_(q);
    const F rho2 = mul_(rho, rho);
    if (flat) {
        ur = mul_(rho2, du);
        ut = mul_(rho2, wn);
        up = mul_(rho2, we);
    } else {
        const F omc = sub_((F)1, tT.y);
        const F Qrr = sub_(omc, mul_(mul_(S.cts, cth), tP.y));
        const F Qrt = fma_(mul_(S.sts, cth), tP.y, tT.x), Qrp = mul_(cth, tP.x);
        const F Qtr = fma_(mul_(sth, S.cts), tP.y, -tT.x);
        const F Qtt = sub_(omc, mul_(mul_(sth, S.sts), tP.y)), Qtp = -mul_(sth, tP.x);
        const F Qpr = -mul_(S.cts, tP.x), Qpt = mul_(S.sts, tP.x), Qpp = sub_((F)1, tP.y);
        ur = mul_(rho2, fma_(Qrr, du, fma_(Qrt, wn, mul_(Qrp, we))));
        ut = mul_(rho2, fma_(Qtr, du, fma_(Qtt, wn, mul_(Qtp, we))));
        up = mul_(rho2, fma_(Qpr, du, fma_(Qpt, wn, mul_(Qpp, we))));
    }
    return mul_(rho, S.inv_s0);  // 1 / T0 = 1 / (s0 sqrt(q))
}

// Lax-Friedrichs update of tau at an interior node for one source (Sec. 3.1 with the
// factor of factor_T0). Dividing the update by T0, with u = p0 / T0 and
// e_d = 1 / (2 delta_d h_d):
//   v = tau_c u + ((tau_d+ - tau_d-) e_d)_d,     H / T0 = sqrt(v^T M v)
//   tau_new = [s / T0 - H / T0 + sum_d c_d (tau_d+ + tau_d-)] / (2 sum_d c_d)
// with c_d = kappa_d e_d, kappa = (1, sqrt(1 - 2 xi), sqrt(1 + 2 xi)): the Cauchy-Schwarz
// bounds of |dH/dp_d| that make the scheme monotone (the Lax-Friedrichs viscosity).
// It is evaluated as an increment of the centre value,
//   tau_new = tau_c + [s / T0 - H / T0 + sum_d c_d ((tau_d+ - tau_c) + (tau_d- - tau_c))]
//                     / (2 sum_d c_d),
// the same value in exact arithmetic. In the direct form the numerator is dominated by the
// neighbour sum (order 2 sum c_d) while the equation's own terms s / T0 - H / T0 are ~100x
// smaller at the benchmark's spacings, so FP32 rounding of that sum acts as a slowness error
// of ~1e-5 and moves the fixed point by ~1.5e-5 of T; the differences to the centre are exact
// (Sterbenz) and small, and the fixed point then sits at FP32's rounding floor.
// trp/trm etc. are tau at the + and - neighbours along r, theta, phi in physical order;
// (invT0, ur, ut, up) are 1/T0 and u, as returned by factor_T0.
template <typename F>
__device__ __forceinline__ F lf_core(F invT0, F ur, F ut, F up, F tc, F trp, F trm, F ttp,
                                     F ttm, F tpp, F tpm, const NodeRec<F> &R, F er) {
    const F vr = fma_(tc, ur, mul_(sub_(trp, trm), er));
    const F vt = fma_(tc, ut, mul_(sub_(ttp, ttm), R.et));
    const F vp = fma_(tc, up, mul_(sub_(tpp, tpm), R.ep));
    const F kt = fma_((F)-2, R.xi, (F)1), kp = fma_((F)2, R.xi, (F)1);
    // q = v_r^2 + (1 - 2 xi) v_t^2 + (1 + 2 xi) v_p^2 + 4 eta v_t v_p
    const F q = fma_(vr, vr, fma_(mul_(kt, vt), vt,
                                  fma_(mul_(kp, vp), vp, mul_(mul_((F)4 * R.eta, vt), vp))));
    const F H = sqrt_(q);
    const F sr = add_(sub_(trp, tc), sub_(trm, tc));
    const F st = add_(sub_(ttp, tc), sub_(ttm, tc));
    const F sp = add_(sub_(tpp, tc), sub_(tpm, tc));
    const F num = fma_(er, sr, fma_(R.ct, st, fma_(R.cp, sp, fma_(R.s, invT0, -H))));
    return fma_(num, R.invW, tc);
}

// Godunov update of tau at an interior node (isotropic models, xi = eta = 0; an alternative to
// lf_core with the same arguments). Along axis d, with e_d = 1 / (delta_d h_d) = 2 x the
// record's half-spacing factor and u the factor's gradient over T0, a one-sided difference
// toward neighbour tau_nb gives the gradient over T0 as a_d tau - b_d, a_d = u_d + sg_d e_d,
// b_d = sg_d e_d tau_nb, sg_d = +1 for the lower neighbour, -1 for the upper. The upwind
// neighbour is the one with the smaller first-order estimate of T: tau_- (e - u) against
// tau_+ (e + u) (both scaled by e / T0_c). tau_new is the smallest root, over the 7
// non-empty subsets of axes, of sum (a_d tau - b_d)^2 = (s / T0)^2 (the larger root of each
// quadratic) whose one-sided differences all keep the upwind sign; with none, tau_c.
// The quadratic is solved for the increment delta = tau - tau_c, with the current one-sided
// gradients c_d = a_d tau_c - b_d = u_d tau_c + sg_d e_d (tau_c - tau_nb): its coefficients
// shrink as the sweep converges, and the larger root is taken in the form without
// cancellation, so FP32 reaches its rounding floor (the direct form of the coefficients
// loses ~1e-5 of tau to cancellation, which the sweeps carry downstream undamped).
template <typename F>
__device__ __forceinline__ F godunov_core(F invT0, F ur, F ut, F up, F tc, F trp, F trm, F ttp,
                                          F ttm, F tpp, F tpm, const NodeRec<F> &R, F er) {
    const F u[3] = {ur, ut, up};
    const F e[3] = {(F)2 * er, (F)2 * R.et, (F)2 * R.ep};
    const F lo[3] = {trm, ttm, tpm}, hi[3] = {trp, ttp, tpp};
    F a[3], c[3], sg[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const bool lower = mul_(lo[d], sub_(e[d], u[d])) <= mul_(hi[d], add_(e[d], u[d]));
        sg[d] = lower ? (F)1 : (F)-1;
        const F se = mul_(sg[d], e[d]);
        a[d] = add_(se, u[d]);
        c[d] = fma_(u[d], tc, mul_(se, sub_(tc, lower ? lo[d] : hi[d])));
    }
    const F rhs = mul_(R.s, invT0);
    const F r2 = mul_(rhs, rhs);
    // Each candidate root is kept as N / D with D > 0: the causality test sg (a N / D + c)
    // >= 0 becomes sg (a N + c D) >= 0 and the comparison of two roots a comparison of
    // cross products, so only the chosen root is divided. A subset's form never exceeds the
    // full one, so a causal root on all three axes is the smallest causal root (the other
    // subsets' quadratics are <= 0 there); the subsets are solved only where it is not.
    {
        F A = 0, B = 0, C = -r2;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            A = fma_(a[d], a[d], A);
            B = fma_(a[d], c[d], B);
            C = fma_(c[d], c[d], C);
        }
        const F disc = fma_(B, B, -mul_(A, C));
        if (A > (F)0 && disc >= (F)0) {
            const F q = sqrt_(disc);
            const bool pos = B >= (F)0;
            const F N = pos ? -C : sub_(q, B);
            const F D = pos ? add_(B, q) : A;
            bool ok = D > (F)0;
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (mul_(sg[d], fma_(a[d], N, mul_(c[d], D))) < (F)0) ok = false;
            if (ok) return add_(tc, div_(N, D));
        }
    }
    F bestN = (F)0, bestD = (F)1;
    bool found = false;
#pragma unroll
    for (int mask = 1; mask < 7; ++mask) {
        F A = 0, B = 0, C = -r2;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (mask >> d & 1) {
                A = fma_(a[d], a[d], A);
                B = fma_(a[d], c[d], B);
                C = fma_(c[d], c[d], C);
            }
        const F disc = fma_(B, B, -mul_(A, C));
        if (!(A > (F)0) || disc < (F)0) continue;
        const F q = sqrt_(disc);
        // the larger root of A delta^2 + 2 B delta + C = 0
        const bool pos = B >= (F)0;
        const F N = pos ? -C : sub_(q, B);
        const F D = pos ? add_(B, q) : A;
        if (!(D > (F)0)) continue;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if ((mask >> d & 1) && mul_(sg[d], fma_(a[d], N, mul_(c[d], D))) < (F)0) ok = false;
        if (ok && (!found || mul_(N, bestD) < mul_(bestN, D))) {
            bestN = N;
            bestD = D;
            found = true;
        }
    }
    return found ? add_(tc, div_(bestN, bestD)) : tc;
}

// Godunov update for anisotropic models (an alternative to lf_core with the same arguments).
// As godunov_core, with two changes. Along theta and phi the upwind neighbour is the side
// the characteristic comes from: the sign of (M g)_d, where g = tau_c u + (tau_+ - tau_-) e_d / 2
// is the central-difference gradient over T0 (the quantity lf_core evaluates). Along r,
// where M has no cross term, it is the neighbour with the smaller estimate of T, as in
// godunov_core. On an axis subset S the components off S take the values that minimise H,
// so the form on S is the Schur complement W = ((M^-1)_SS)^-1:
//   {r}: 1; {theta}: det / m_p; {phi}: det / m_t; {r, theta}, {r, phi}: diagonal;
//   {theta, phi}: the (theta, phi) block of M; {r, theta, phi}: M,
// with m_t = 1 - 2 xi, m_p = 1 + 2 xi, m = 2 eta, det = m_t m_p - m^2. The 1-D and diagonal
// quadratics are scaled by m_p or m_t (> 0), which leaves their roots and signs unchanged and
// needs no division. Causality: sg_d (W g)_d >= 0 on S. Increment form and division-free
// selection as in godunov_core.
template <typename F>
__device__ __forceinline__ F godunov_aniso_core(F invT0, F ur, F ut, F up, F tc, F trp, F trm,
                                                F ttp, F ttm, F tpp, F tpm, const NodeRec<F> &R,
                                                F er) {
    const F u[3] = {ur, ut, up};
    const F eh[3] = {er, R.et, R.ep};
    const F lo[3] = {trm, ttm, tpm}, hi[3] = {trp, ttp, tpp};
    const F mt = fma_((F)-2, R.xi, (F)1), mp = fma_((F)2, R.xi, (F)1), m = (F)2 * R.eta;
    const F det = fma_(mt, mp, -mul_(m, m));
    F gc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) gc[d] = fma_(tc, u[d], mul_(sub_(hi[d], lo[d]), eh[d]));
    bool lower[3];
    {
        const F e0 = (F)2 * eh[0];
        lower[0] = mul_(lo[0], sub_(e0, u[0])) <= mul_(hi[0], add_(e0, u[0]));
        lower[1] = fma_(mt, gc[1], mul_(m, gc[2])) >= (F)0;
        lower[2] = fma_(m, gc[1], mul_(mp, gc[2])) >= (F)0;
    }
    F a[3], c[3], sg[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        sg[d] = lower[d] ? (F)1 : (F)-1;
        const F se = mul_(sg[d], (F)2 * eh[d]);
        a[d] = add_(se, u[d]);
        c[d] = fma_(u[d], tc, mul_(se, sub_(tc, lower[d] ? lo[d] : hi[d])));
    }
    const F rhs = mul_(R.s, invT0);
    const F r2 = mul_(rhs, rhs);
    // per-axis products shared by the subsets
    const F aa0 = mul_(a[0], a[0]), ac0 = mul_(a[0], c[0]), cc0 = mul_(c[0], c[0]);
    const F aa1 = mul_(a[1], a[1]), ac1 = mul_(a[1], c[1]), cc1 = mul_(c[1], c[1]);
    const F aa2 = mul_(a[2], a[2]), ac2 = mul_(a[2], c[2]), cc2 = mul_(c[2], c[2]);
    // the (theta, phi) block form
    const F Atp = fma_(mt, aa1, fma_(mul_((F)2 * m, a[1]), a[2], mul_(mp, aa2)));
    const F Btp = fma_(mt, ac1, fma_(m, fma_(a[1], c[2], mul_(a[2], c[1])), mul_(mp, ac2)));
    const F Ctp = fma_(mt, cc1, fma_(mul_((F)2 * m, c[1]), c[2], mul_(mp, cc2)));
    // The form on a subset S is the minimum of the full form over the components off S, so
    // it never exceeds the full form: at a causal 3-D root tau* every subset's quadratic is
    // <= 0 and its larger root >= tau*. A causal 3-D root is therefore the answer, and the
    // other subsets are solved only where it is not causal.
    {
        const F A = add_(aa0, Atp), B = add_(ac0, Btp), C = sub_(add_(cc0, Ctp), r2);
        const F disc = fma_(B, B, -mul_(A, C));
        if (A > (F)0 && disc >= (F)0) {
            const F q = sqrt_(disc);
            const bool pos = B >= (F)0;
            const F N = pos ? -C : sub_(q, B);
            const F D = pos ? add_(B, q) : A;
            const F h0 = fma_(a[0], N, mul_(c[0], D));
            const F h1 = fma_(a[1], N, mul_(c[1], D));
            const F h2 = fma_(a[2], N, mul_(c[2], D));
            if (D > (F)0 && mul_(sg[0], h0) >= (F)0 &&
                mul_(sg[1], fma_(mt, h1, mul_(m, h2))) >= (F)0 &&
                mul_(sg[2], fma_(m, h1, mul_(mp, h2))) >= (F)0)
                return add_(tc, div_(N, D));
        }
    }
    // One axis subset (bit 0 r, bit 1 theta, bit 2 phi): its root as N / D and whether it is
    // valid and causal.
    auto cand = [&](const int mask, F &N, F &D) -> bool {
        const bool hr = mask & 1, ht = mask & 2, hp = mask & 4;
        F A, B, C;
        if (ht && hp) {
            A = hr ? add_(aa0, Atp) : Atp;
            B = hr ? add_(ac0, Btp) : Btp;
            C = sub_(hr ? add_(cc0, Ctp) : Ctp, r2);
        } else if (ht || hp) {
            const F sc = ht ? mp : mt;               // scale of the 1-D theta / phi form
            const F aa = ht ? aa1 : aa2, ac = ht ? ac1 : ac2, cc = ht ? cc1 : cc2;
            A = hr ? fma_(sc, aa0, mul_(det, aa)) : mul_(det, aa);
            B = hr ? fma_(sc, ac0, mul_(det, ac)) : mul_(det, ac);
            C = hr ? fma_(sc, cc0, fma_(det, cc, -mul_(sc, r2))) : fma_(det, cc, -mul_(sc, r2));
        } else {
            A = aa0;
            B = ac0;
            C = sub_(cc0, r2);
        }
        const F disc = fma_(B, B, -mul_(A, C));
        if (!(A > (F)0) || disc < (F)0) return false;
        const F q = sqrt_(disc);
        const bool pos = B >= (F)0;
        N = pos ? -C : sub_(q, B);
        D = pos ? add_(B, q) : A;
        if (!(D > (F)0)) return false;
        // D (a delta + c) on each axis, then the causality test on W g
        const F h0 = fma_(a[0], N, mul_(c[0], D));
        const F h1 = fma_(a[1], N, mul_(c[1], D));
        const F h2 = fma_(a[2], N, mul_(c[2], D));
        bool ok = !hr || mul_(sg[0], h0) >= (F)0;
        if (ht && hp) {
            ok = ok && mul_(sg[1], fma_(mt, h1, mul_(m, h2))) >= (F)0 &&
                 mul_(sg[2], fma_(m, h1, mul_(mp, h2))) >= (F)0;
        } else if (ht) {
            ok = ok && mul_(sg[1], h1) >= (F)0;
        } else if (hp) {
            ok = ok && mul_(sg[2], h2) >= (F)0;
        }
        return ok;
    };
    F bestN = (F)0, bestD = (F)1;
    bool found = false;
    auto take = [&](const F N, const F D) {
        if (!found || mul_(N, bestD) < mul_(bestN, D)) {
            bestN = N;
            bestD = D;
            found = true;
        }
    };
    F N, D;
    const bool ok3 = cand(3, N, D);
    if (ok3) take(N, D);
    const bool ok5 = cand(5, N, D);
    if (ok5) take(N, D);
    const bool ok6 = cand(6, N, D);
    if (ok6) take(N, D);
    // By the same argument a causal root on two axes is no larger than the roots on either
    // of its single axes, so a single axis is solved only where neither pair holding it is
    // causal.
    if (!ok3 && !ok5 && cand(1, N, D)) take(N, D);
    if (!ok3 && !ok6 && cand(2, N, D)) take(N, D);
    if (!ok5 && !ok6 && cand(4, N, D)) take(N, D);
    return found ? add_(tc, div_(bestN, bestD)) : tc;
}

// ---------------------------------------------------------------------------------------
// Grid-wide barrier for persistent cooperative launches. Arrivals go to a monotonic
// per-launch counter: barrier number m of a launch is complete once m * nblocks arrivals
// have been counted, so a barrier costs one acquire-release fence, one fire-and-forget
// atomic and the polling of one L2 line (the status word, on the same line, is read with
// the first poll). Every wait is bounded by a deadline on the global nanosecond timer; on expiry
// the status word gets kDevTimeout and the caller returns. All blocks eventually leave: a
// block that gave up never arrives again, so the others' waits expire too. The status word
// is sticky, so later launches of the same solve stop at their first barrier.
struct alignas(128) BarrierState {  // one L2 line per barrier group
    unsigned long long arrived;     // arrivals since the launch started
    unsigned int left;              // blocks that have finished the launch
    int status;
    int pad[28];
};

// Arrivals the calling block waits for at its next barrier (read and written by thread 0).
static __shared__ unsigned long long s_bar_target;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_relaxed_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ int ld_status(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Called by every block of a launch before its first barrier.
__device__ __forceinline__ void barrier_begin() {
    if (threadIdx.x == 0) s_bar_target = 0;
}

// Returns false when the barrier (or an earlier one in another block) timed out. nblocks is
// the number of blocks that take part (all blocks of the launch, or one barrier group).
__device__ __forceinline__ bool grid_barrier(BarrierState *bs, unsigned long long limit_ns,
                                             unsigned int nblocks) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        const unsigned long long target = s_bar_target + nblocks;
        s_bar_target = target;
        // release: the fence orders the block's writes (made visible to this thread by
        // __syncthreads) before the arrival; the acquiring load below pairs with the other
        // blocks' fences, and __syncthreads passes the ordering on to the whole block
        fence_acq_rel_gpu();
        red_relaxed_add(&bs->arrived, 1ull);
        // another block's timeout, read together with the first poll rather than after the
        // wait, so that it adds no round trip to the barrier (a timeout during this wait is
        // then seen at the next barrier, which the block that timed out never reaches)
        const int st0 = ld_status(&bs->status);
        if (ld_acquire(&bs->arrived) < target) {
            if (st0 != 0) good = 0;  // a block gave up earlier: no one waits for it
            const unsigned long long t0 = global_ns();
            unsigned int ns = 16;
            while (good && ld_acquire(&bs->arrived) < target) {
                if (global_ns() - t0 > limit_ns) {
                    atomicExch(&bs->status, (int)kDevTimeout);
                    good = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 64) ns <<= 1;
            }
        }
        if (good && st0 != 0) good = 0;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ bool grid_barrier(BarrierState *bs, unsigned long long limit_ns) {
    return grid_barrier(bs, limit_ns, gridDim.x);
}

// Called by every block that reached the normal end of the launch: the last one to leave
// clears the counters, so that the next launch on the same words starts from zero (launches
// on one stream do not overlap).
__device__ __forceinline__ void barrier_end(BarrierState *bs, unsigned int nblocks) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&bs->left, 1u) == nblocks - 1) {
            atomicExch(&bs->arrived, 0ull);
            atomicExch(&bs->left, 0u);
        }
    }
}

}  // namespace ttgb
