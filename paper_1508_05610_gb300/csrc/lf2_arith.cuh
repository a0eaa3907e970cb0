// lf2_arith.cuh -- the device arithmetic every leapfrog kernel of liblf2 compiles: coefficient
// packs, the per-site update functions and the lattice geometry helpers.
//
// Every kernel variant (one thread per site, z-streaming tiles, temporal blocking, ensemble)
// performs the per-site update through the functions below, written with explicit
// round-to-nearest intrinsics so that the compiler cannot contract or reorder them
// differently in different kernels: all variants give bitwise identical results.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lf2.h"

namespace lf2 {

constexpr int kMaxComp = LF2_MAX_COMP;

// ---------------------------------------------------------------- coefficient packs
// FP64: the force enters only through dt*F, folded as
//   dt F_a = a * nb_a - (dl * s2 + b0) * phi_a
// with nb_a the sum of the 6 neighbours, s2 = sum_b phi_b^2 and
//   a = dt/dx^2,  dl = dt lambda,  b0 = dt (6/dx^2 + m2 - lambda eta^2).
struct Coef64 {
    double a, dl, b0, dt;
};

// FP32: difference form of the Laplacian (sum_i (phi(x+-i) - phi(x))), which keeps the
// small differences of a smooth field exact when |phi| ~ eta, then
//   F_a = d_a * inv_dx2 - (lambda (s2 - eta^2) + m2) phi_a.
struct Coef32 {
    float inv_dx2, lam, eta2, m2, dt;
    float zero;  // always 0: a run-time zero for the packed path (see make_coef32x2)
};

// Energy (always FP64).  The synchronised momentum pi_n = pi_{n-1/2} + (dt/2) F(phi_n) is a
// kick of half a step, folded as in Coef64 with dt/2: ah = (dt/2)/dx^2, hl = (dt/2) lambda,
// hb0 = (dt/2)(6/dx^2 + m2 - lambda eta^2).  The remaining members scale the raw sums.
struct CoefE {
    double ah, hl, hb0, eta2;
    double inv_dx2, lam, m2, vol;  // vol = dx^3
};

inline Coef64 make_coef64(const lf2_params &p, double dt) {
    const double inv_dx2 = 1.0 / (p.dx * p.dx);
    return Coef64{dt * inv_dx2, dt * p.lambda, dt * (6.0 * inv_dx2 + p.m2 - p.lambda * p.eta * p.eta), dt};
}

inline Coef32 make_coef32(const lf2_params &p, double dt) {
    return Coef32{(float)(1.0 / (p.dx * p.dx)), (float)p.lambda, (float)(p.eta * p.eta), (float)p.m2, (float)dt, 0.0f};
}

inline CoefE make_coefE(const lf2_params &p) {
    const double inv_dx2 = 1.0 / (p.dx * p.dx), h = 0.5 * p.dt;
    return CoefE{h * inv_dx2, h * p.lambda, h * (6.0 * inv_dx2 + p.m2 - p.lambda * p.eta * p.eta), p.eta * p.eta,
                 inv_dx2,     p.lambda,     p.m2,                                                   p.dx * p.dx * p.dx};
}

// ------------------------------------------------------------------ per-site update
// Neighbour values are passed in the fixed order -x, +x, -y, +y, -z, +z.

// FP64 kick (+ drift).  pi <- pi + dt F(phi);  phi_out <- phi + dt pi.
template <int NC>
__device__ __forceinline__ void update_f64(const double (&c)[NC], const double (&xm)[NC], const double (&xp)[NC],
                                           const double (&ym)[NC], const double (&yp)[NC], const double (&zm)[NC],
                                           const double (&zp)[NC], double (&p)[NC], double (&out)[NC],
                                           const Coef64 &k) {
    double s2 = __dmul_rn(c[0], c[0]);
#pragma unroll
    for (int b = 1; b < NC; ++b) s2 = __fma_rn(c[b], c[b], s2);
    const double g = __fma_rn(k.dl, s2, k.b0);
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        // neighbour sum as a tree (depth 3 instead of a chain of 5 dependent adds)
        const double nb = __dadd_rn(__dadd_rn(xm[a], xp[a]), __dadd_rn(__dadd_rn(ym[a], yp[a]), __dadd_rn(zm[a], zp[a])));
        p[a] = __fma_rn(k.a, nb, __fma_rn(-g, c[a], p[a]));
        out[a] = __fma_rn(k.dt, p[a], c[a]);
    }
}

// FP32 force, difference form.
template <int NC>
__device__ __forceinline__ void force_f32(const float (&c)[NC], const float (&xm)[NC], const float (&xp)[NC],
                                          const float (&ym)[NC], const float (&yp)[NC], const float (&zm)[NC],
                                          const float (&zp)[NC], float (&F)[NC], const Coef32 &k) {
    float s2 = __fmul_rn(c[0], c[0]);
#pragma unroll
    for (int b = 1; b < NC; ++b) s2 = __fmaf_rn(c[b], c[b], s2);
    const float g = __fmaf_rn(k.lam, __fsub_rn(s2, k.eta2), k.m2);
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        const float dx_ = __fadd_rn(__fsub_rn(xm[a], c[a]), __fsub_rn(xp[a], c[a]));
        const float dy_ = __fadd_rn(__fsub_rn(ym[a], c[a]), __fsub_rn(yp[a], c[a]));
        const float dz_ = __fadd_rn(__fsub_rn(zm[a], c[a]), __fsub_rn(zp[a], c[a]));
        const float d = __fadd_rn(__fadd_rn(dx_, dy_), dz_);
        F[a] = __fmaf_rn(d, k.inv_dx2, -__fmul_rn(g, c[a]));
    }
}

// FP32 kick + drift; KAHAN selects the compensated drift
//   y = dt pi - comp;  t = phi + y;  comp = (t - phi) - y;  phi_out = t.
template <int NC, bool KAHAN>
__device__ __forceinline__ void update_f32(const float (&c)[NC], const float (&xm)[NC], const float (&xp)[NC],
                                           const float (&ym)[NC], const float (&yp)[NC], const float (&zm)[NC],
                                           const float (&zp)[NC], float (&p)[NC], float (&cmp)[NC],
                                           float (&out)[NC], const Coef32 &k) {
    float F[NC];
    force_f32<NC>(c, xm, xp, ym, yp, zm, zp, F, k);
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        p[a] = __fmaf_rn(k.dt, F[a], p[a]);
        if (KAHAN) {
            const float y = __fmaf_rn(k.dt, p[a], -cmp[a]);
            const float t = __fadd_rn(c[a], y);
            cmp[a] = __fsub_rn(__fsub_rn(t, c[a]), y);
            out[a] = t;
        } else {
            out[a] = __fmaf_rn(k.dt, p[a], c[a]);
        }
    }
}

// FP64 kick only (start of the staggered scheme): pi <- pi + dt' F(phi).
template <int NC>
__device__ __forceinline__ void kick_f64(const double (&c)[NC], const double (&xm)[NC], const double (&xp)[NC],
                                         const double (&ym)[NC], const double (&yp)[NC], const double (&zm)[NC],
                                         const double (&zp)[NC], double (&p)[NC], const Coef64 &k) {
    double out[NC];
    update_f64<NC>(c, xm, xp, ym, yp, zm, zp, p, out, k);
}

template <int NC>
__device__ __forceinline__ void kick_f32(const float (&c)[NC], const float (&xm)[NC], const float (&xp)[NC],
                                         const float (&ym)[NC], const float (&yp)[NC], const float (&zm)[NC],
                                         const float (&zp)[NC], float (&p)[NC], const Coef32 &k) {
    float F[NC];
    force_f32<NC>(c, xm, xp, ym, yp, zm, zp, F, k);
#pragma unroll
    for (int a = 0; a < NC; ++a) p[a] = __fmaf_rn(k.dt, F[a], p[a]);
}

// ------------------------------------------------------- packed FP32 pairs (f32x2)
// Two sites updated by one instruction stream with Blackwell's packed f32x2 arithmetic.
// Each lane is an IEEE round-to-nearest FP32 operation, and the sequence below is the one of
// force_f32 / update_f32 rewritten with exact sign identities of round-to-nearest
// (RN(-a*b - c) = -RN(a*b + c)), so a packed update is bitwise equal to two scalar ones.
// One caution, found by measurement: the assembler may fuse a packed multiply whose result
// feeds a packed add or subtract into a single fused multiply-add (one rounding instead of
// two) even with explicit .rn.  No product below feeds an add: c*c is formed as
// fma(c, c, zero) with a zero the compiler cannot see (RN(c*c + 0) = RN(c*c) for every c),
// and the other products feed the addend of an fma, which cannot be fused further.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(f32x2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Coefficients broadcast to both lanes; n* are negated copies.
struct Coef32x2 {
    f32x2 inv_dx2, nlam, eta2, nm2, dt, ndt, zero;
};

// `zero` must be a run-time 0 (the caller passes a kernel argument), never a literal.
__device__ __forceinline__ Coef32x2 make_coef32x2(const Coef32 &k, float zero) {
    return Coef32x2{pk2(k.inv_dx2, k.inv_dx2), pk2(-k.lam, -k.lam), pk2(k.eta2, k.eta2), pk2(-k.m2, -k.m2),
                    pk2(k.dt, k.dt),           pk2(-k.dt, -k.dt),   pk2(zero, zero)};
}

// update_f32 for two sites at once (lane 0 and lane 1 of every operand).
template <int NC, bool KAHAN>
__device__ __forceinline__ void update_f32x2(const f32x2 (&c)[NC], const f32x2 (&xm)[NC], const f32x2 (&xp)[NC],
                                             const f32x2 (&ym)[NC], const f32x2 (&yp)[NC], const f32x2 (&zm)[NC],
                                             const f32x2 (&zp)[NC], f32x2 (&p)[NC], f32x2 (&cmp)[NC],
                                             f32x2 (&out)[NC], const Coef32x2 &k) {
    f32x2 s2 = fma2(c[0], c[0], k.zero);
#pragma unroll
    for (int b = 1; b < NC; ++b) s2 = fma2(c[b], c[b], s2);
    const f32x2 ng = fma2(k.nlam, sub2(s2, k.eta2), k.nm2);  // -g
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        const f32x2 dx_ = add2(sub2(xm[a], c[a]), sub2(xp[a], c[a]));
        const f32x2 dy_ = add2(sub2(ym[a], c[a]), sub2(yp[a], c[a]));
        const f32x2 dz_ = add2(sub2(zm[a], c[a]), sub2(zp[a], c[a]));
        const f32x2 d = add2(add2(dx_, dy_), dz_);
        const f32x2 F = fma2(d, k.inv_dx2, mul2(ng, c[a]));  // d/dx^2 - g c
        p[a] = fma2(k.dt, F, p[a]);
        if (KAHAN) {
            const f32x2 ny = fma2(k.ndt, p[a], cmp[a]);  // -(dt p - comp)
            const f32x2 t = sub2(c[a], ny);
            cmp[a] = add2(sub2(t, c[a]), ny);
            out[a] = t;
        } else {
            out[a] = fma2(k.dt, p[a], c[a]);
        }
    }
}

// update_f32 for one two-component site, its components packed as one f32x2 pair (the
// interleaved storage order): |phi|^2 and the potential coefficient are formed in scalar
// exactly as force_f32 does, everything per component runs packed.
template <bool KAHAN>
__device__ __forceinline__ void update_f32_site2(f32x2 c, f32x2 xm, f32x2 xp, f32x2 ym, f32x2 yp, f32x2 zm, f32x2 zp,
                                                 f32x2 &p, f32x2 &cmp, f32x2 &out, const Coef32x2 &k,
                                                 const Coef32 &ks) {
    float c0, c1;
    up2(c, c0, c1);
    const float s2 = __fmaf_rn(c1, c1, __fmul_rn(c0, c0));
    const float ngs = __fmaf_rn(-ks.lam, __fsub_rn(s2, ks.eta2), -ks.m2);  // -g
    const f32x2 ng = pk2(ngs, ngs);
    const f32x2 dx_ = add2(sub2(xm, c), sub2(xp, c));
    const f32x2 dy_ = add2(sub2(ym, c), sub2(yp, c));
    const f32x2 dz_ = add2(sub2(zm, c), sub2(zp, c));
    const f32x2 d = add2(add2(dx_, dy_), dz_);
    const f32x2 F = fma2(d, k.inv_dx2, mul2(ng, c));
    p = fma2(k.dt, F, p);
    if (KAHAN) {
        const f32x2 ny = fma2(k.ndt, p, cmp);
        const f32x2 t = sub2(c, ny);
        cmp = add2(sub2(t, c), ny);
        out = t;
    } else {
        out = fma2(k.dt, p, c);
    }
}

// update_f32 for one site of NC >= 3 components: |phi|^2 and the potential coefficient in
// scalar exactly as force_f32 forms them, the components in packed pairs (0,1), (2,3), ...
// with update_f32_site2's per-component sequence, and an odd last component in scalar with
// update_f32's own sequence (-g c = RN(ng * c) since ng = -g exactly).
template <int NC, bool KAHAN>
__device__ __forceinline__ void update_f32_siteN(const float (&c)[NC], const float (&xm)[NC], const float (&xp)[NC],
                                                 const float (&ym)[NC], const float (&yp)[NC], const float (&zm)[NC],
                                                 const float (&zp)[NC], float (&p)[NC], float (&cmp)[NC],
                                                 float (&out)[NC], const Coef32x2 &k, const Coef32 &ks) {
    float s2 = __fmul_rn(c[0], c[0]);
#pragma unroll
    for (int b = 1; b < NC; ++b) s2 = __fmaf_rn(c[b], c[b], s2);
    const float ngs = __fmaf_rn(-ks.lam, __fsub_rn(s2, ks.eta2), -ks.m2);  // -g
    const f32x2 ng = pk2(ngs, ngs);
#pragma unroll
    for (int q = 0; q < NC / 2; ++q) {
        const int a0 = 2 * q, a1 = 2 * q + 1;
        const f32x2 C = pk2(c[a0], c[a1]);
        const f32x2 dx_ = add2(sub2(pk2(xm[a0], xm[a1]), C), sub2(pk2(xp[a0], xp[a1]), C));
        const f32x2 dy_ = add2(sub2(pk2(ym[a0], ym[a1]), C), sub2(pk2(yp[a0], yp[a1]), C));
        const f32x2 dz_ = add2(sub2(pk2(zm[a0], zm[a1]), C), sub2(pk2(zp[a0], zp[a1]), C));
        const f32x2 d = add2(add2(dx_, dy_), dz_);
        const f32x2 F = fma2(d, k.inv_dx2, mul2(ng, C));
        f32x2 P = fma2(k.dt, F, pk2(p[a0], p[a1]));
        f32x2 O;
        if (KAHAN) {
            const f32x2 ny = fma2(k.ndt, P, pk2(cmp[a0], cmp[a1]));
            const f32x2 t = sub2(C, ny);
            up2(add2(sub2(t, C), ny), cmp[a0], cmp[a1]);
            O = t;
        } else {
            O = fma2(k.dt, P, C);
        }
        up2(P, p[a0], p[a1]);
        up2(O, out[a0], out[a1]);
    }
    if constexpr (NC % 2 == 1) {
        constexpr int a = NC - 1;
        const float dx_ = __fadd_rn(__fsub_rn(xm[a], c[a]), __fsub_rn(xp[a], c[a]));
        const float dy_ = __fadd_rn(__fsub_rn(ym[a], c[a]), __fsub_rn(yp[a], c[a]));
        const float dz_ = __fadd_rn(__fsub_rn(zm[a], c[a]), __fsub_rn(zp[a], c[a]));
        const float d = __fadd_rn(__fadd_rn(dx_, dy_), dz_);
        const float F = __fmaf_rn(d, ks.inv_dx2, __fmul_rn(ngs, c[a]));
        p[a] = __fmaf_rn(ks.dt, F, p[a]);
        if (KAHAN) {
            const float y = __fmaf_rn(ks.dt, p[a], -cmp[a]);
            const float t = __fadd_rn(c[a], y);
            cmp[a] = __fsub_rn(__fsub_rn(t, c[a]), y);
            out[a] = t;
        } else {
            out[a] = __fmaf_rn(ks.dt, p[a], c[a]);
        }
    }
}

// ----------------------------------------------------------------- geometry helpers
struct Geom {
    int nx, ny, nz;
    long long sites;
};

__device__ __forceinline__ int wrap_dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int wrap_up(int i, int n) { return i == n - 1 ? 0 : i + 1; }

}  // namespace lf2
