// pt_device.cuh -- device-side building blocks of the transit-model kernels.
//
// Everything here is FP32 except where a comment says otherwise.  The
// numerical choices are documented next to the code; the formulas follow
// Parviainen (2015) Sec. 2.2.1, Eq. (ma_model), with the lambda/eta functions
// of Mandel & Agol (2002), which the paper defers to.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define PT_PI_F 3.14159265358979f
#define PT_ZBEHIND 1.0e30f

namespace pt {

// ---------------------------------------------------------------------------
// Per-geometry record, written by the set-up kernel and staged in shared
// memory by the light-curve kernels.  One record per (vector) or, when every
// passband has its own radius ratio, per (vector, passband).
//
// Time is reduced in double-float arithmetic: t0 and P are split into a
// high float and the float of the remainder, so that t - t0 - n P keeps
// ~1e-11 d absolute accuracy at |t| ~ 1e3 d without FP64 instructions on the
// hot path.  The eccentric-orbit anchor (the eccentric anomaly at
// conjunction) is computed in FP64 by the set-up kernel and enters the hot
// path only multiplied by small quantities (see orbit_z below).
// ---------------------------------------------------------------------------
struct __align__(16) GeomRec {
    float t0h, t0l, Ph, Pl;   // double-float t0 and P
    float invP, nang;         // 1/P, 2 pi / P
    float win_lo, win_hi;     // transit window in (t - t0 - nP) [days]; empty if lo > hi
    float a, cosi, k, ecc;    // a/R*, cos i, radius ratio, 0 = circular / 1 = eccentric
    float ecE, esE, cE, sE;   // e cos E_tr, e sin E_tr, cos E_tr, sin E_tr
    float Uc, Us, Vs, Vc;     // a cos w, a sqrt(1-e^2) sin w, a sin w, a sqrt(1-e^2) cos w
    float Vtr, nq, pad1, pad2;    // r at conjunction = a (1 - e cos E_tr); e / (1 - e) (Newton's error factor)
};
static_assert(sizeof(GeomRec) == 96, "GeomRec layout");

// t - t0 - n P for the nearest epoch n, in double-float arithmetic.
// (th, tl) is the double-float split of t.  Two-sum error terms are exact.
__device__ __forceinline__ float reduce_time(float th, float tl, const GeomRec &r)
{
    float s = th - r.t0h;
    float bv = s - th;
    float e1 = (th - (s - bv)) + (-r.t0h - bv);
    float n = rintf(s * r.invP);
    float p = n * r.Ph;
    float pe = fmaf(n, r.Ph, -p);          // n*Ph = p + pe exactly
    float d = s - p;
    float bv2 = d - s;
    float e2 = (s - (d - bv2)) + (-p - bv2);
    float lo = ((e1 + e2) - pe) + (tl - r.t0l) - n * r.Pl;
    return d + lo;
}

// One-instruction hardware approximations (PTX rcp.approx.ftz, sqrt.approx.ftz:
// about one ulp, denormal inputs and results flushed to zero).  Without the
// .ftz form each call also carries the scaling that handles denormals.  The
// Mandel-Agol core uses them only where its arguments are normal numbers or
// exact zeros by construction (stated at each use).
__device__ __forceinline__ float rcp_a(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_a(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// atan2(y, x) for y >= 0 (an angle in [0, pi]), for the lens angles of the
// Mandel-Agol terms.  r = min(y, |x|) / max(y, |x|) lies in [0, 1] and
// atan(r) = r P(r^2) with P of degree 8, fitted to atan(r)/r on [0, 1] by
// Lawson's iteratively reweighted least squares (towards the minimax fit;
// csrc/atan_poly.py recomputes the coefficients): 1.4e-8 absolute in FP64,
// about 1.2e-7 evaluated in FP32.  Then atan2 = pi/2 - atan(r) when y > |x|,
// and pi minus that when x < 0.  Both arguments zero give 0.
__device__ __forceinline__ float atan2_pos(float y, float x)
{
    const float ax = fabsf(x);
    const float mx = fmaxf(y, ax), mn = fminf(y, ax);
    const float r = mx > 0.0f ? mn * rcp_a(mx) : 0.0f;   // mx is 0 or a normal number here
    const float s = r * r;
    float q = 2.903584391e-03f;
    q = fmaf(q, s, -1.628314145e-02f);
    q = fmaf(q, s, 4.303959757e-02f);
    q = fmaf(q, s, -7.533697039e-02f);
    q = fmaf(q, s, 1.065468788e-01f);
    q = fmaf(q, s, -1.420713663e-01f);
    q = fmaf(q, s, 1.999305487e-01f);
    q = fmaf(q, s, -3.333309293e-01f);
    q = fmaf(q, s, 1.0f);
    float t = r * q;
    if (y > ax) t = 0.5f * PT_PI_F - t;
    if (x < 0.0f) t = PT_PI_F - t;
    return t;
}

// First pass of the window test, in plain FP32: false only when t - t0 - nP
// is certainly outside [win_lo, win_hi].  One FMA does the reduction with
// the same epoch n as reduce_time; against the double-float result it drops
// the rounding of s, the low parts of t, t0 and P and rounds once more, so
// it is off by less than 2^-24 (|s| + |t_h| + |t0_h| + |n| P_h + |d|); the
// margin doubles that (plus a nanosecond-scale floor).
__device__ __forceinline__ bool maybe_in_window(float th, const GeomRec &r)
{
    float s = th - r.t0h;
    float n = rintf(s * r.invP);
    float d = fmaf(-n, r.Ph, s);
    float m = 1.2e-7f * (fabsf(s) + fabsf(th) + fabsf(r.t0h) + fabsf(n) * r.Ph + fabsf(d)) + 1e-9f;
    return (d + m >= r.win_lo) && (d - m <= r.win_hi);
}

// sin h and cos h by their Taylor series through h^9 and h^10, for the
// small angles of the transit window (|h| <= 0.4: the first omitted terms,
// h^11/11! and h^12/12!, are below 1e-11 relative); other angles take
// sincosf.
__device__ __forceinline__ void sincos_near0(float h, float *s, float *c)
{
    if (fabsf(h) <= 0.4f) {
        const float h2 = h * h;
        float ps = fmaf(h2, 1.0f / 362880.0f, -1.0f / 5040.0f);
        ps = fmaf(h2, ps, 1.0f / 120.0f);
        ps = fmaf(h2, ps, -1.0f / 6.0f);
        *s = fmaf(h * h2, ps, h);
        float pc = fmaf(h2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
        pc = fmaf(h2, pc, -1.0f / 720.0f);
        pc = fmaf(h2, pc, 1.0f / 24.0f);
        pc = fmaf(h2, pc, -0.5f);
        *c = fmaf(h2, pc, 1.0f);
    } else {
        sincosf(h, s, c);
    }
}

// Projected separation z at time offset dt from conjunction (Sec. 1; the
// paper prints no orbit formula).
//   Circular:  phi = 2 pi dt / P,  z = a sqrt(sin^2 phi + cos^2 i cos^2 phi).
//   Eccentric: Kepler's equation is solved relative to the conjunction
//     anchor E_tr (M_tr = E_tr - e sin E_tr):
//       dE - e cos E_tr sin dE + e sin E_tr (1 - cos dE) = dM,  dM = 2 pi dt / P,
//     by Newton's method.  Position in the sky plane relative to conjunction:
//       U = r cos(w + f) = a cos w dC - a sqrt(1-e^2) sin w dS        (U_tr = 0)
//       V = r sin(w + f) = V_tr + a sin w dC + a sqrt(1-e^2) cos w dS
//     with dC = cos E - cos E_tr, dS = sin E - sin E_tr formed from sin dE and
//     1 - cos dE = 2 sin^2(dE/2).  Every term is small near transit, so FP32
//     keeps relative accuracy there; z = sqrt(U^2 + V^2 cos^2 i).
//   Behind the star (cos phi <= 0, or V <= 0) returns PT_ZBEHIND.
// Newton stops once the error left after a step, at most (e / (2 (1 - e)))
// step^2 (|f''| <= e, f' >= 1 - e for this f), is below 3e-8 |dE|: the
// rounding level of the FP32 evaluation, so no step is spent on merely
// confirming convergence.  *bad is set when that did not happen within
// max_iter steps.
// Warm start: a caller stepping through the supersamples of one exposure
// passes warm[3] = {dE, dM, dE/dM} of the previous solution (warm[0] NaN for
// none); the start dE + (dM' - dM) dE/dM is then off by ~e (dM' - dM)^2 / 2,
// so one Newton step usually converges.  The solution is written back.
// FAST takes the Newton quotient with the one-instruction reciprocal (its
// denominator 1 - e cos E lies in [1 - e, 1 + e]) and the final root with the
// one-instruction square root (an argument below 2^-126, a separation under
// 1e-19, gives 0): about one ulp more in z.  ROT takes sin and cos of dE/2 at the solution
// from the last step's values (below) instead of a second series; the
// per-supersample loops of the pair-list kernels gain from it, while in the
// batched and tile kernels the extra live values cost more than the series.
template <bool FAST = false, bool ROT = false>
__device__ __forceinline__ float orbit_z(const GeomRec &r, float dt, int max_iter, bool *bad, float *warm = nullptr)
{
    if (r.ecc == 0.0f) {
        float s, c;
        sincos_near0(r.nang * dt, &s, &c);
        if (c <= 0.0f) return PT_ZBEHIND;
        float ci = r.cosi * c;
        return r.a * (FAST ? sqrt_a(fmaf(s, s, ci * ci)) : sqrtf(fmaf(s, s, ci * ci)));
    }
    float dM = r.nang * dt;
    float dE = (warm && warm[0] == warm[0]) ? fmaf(dM - warm[1], warm[2], warm[0]) : dM / (1.0f - r.ecE);
    float sh = 0.0f, ch = 1.0f, dEdM = 1.0f, step = 0.0f;
    bool conv = false;
    for (int it = 0; it < max_iter; ++it) {
        sincos_near0(0.5f * dE, &sh, &ch);
        float sn = 2.0f * sh * ch, omc = 2.0f * sh * sh;
        float F = (dE - r.ecE * sn) + (r.esE * omc - dM);
        float Fp = 1.0f - r.ecE * (1.0f - omc) + r.esE * sn;
        if (FAST) {
            dEdM = rcp_a(Fp);
            step = F * dEdM;
        } else {
            step = F / Fp;
            if (warm) dEdM = __fdividef(1.0f, Fp);
        }
        dE -= step;
        if (r.nq * step * step <= 6e-8f * fabsf(dE) + 1e-12f) {
            conv = true;
            break;
        }
    }
    if (!conv) *bad = true;
    if (warm) {
        warm[0] = dE;
        warm[1] = dM;
        warm[2] = dEdM;
    }
    if (ROT) {
        // sin and cos of dE/2 at the solution: the last step's values rotated
        // by -step/2 with cos(step/2) ~ 1 - step^2/8, sin(step/2) ~ step/2.
        // The dropped terms are third order in step/2: the stopping rule
        // accepts |step| <= sqrt(6e-8 |dE| / nq) (< 1e-3 unless e is tiny,
        // where the Newton step itself is at most e |dM|), so they stay
        // below 1e-10.
        const float h = 0.5f * step;
        const float c = fmaf(-0.5f * h, h, 1.0f);
        const float sh1 = fmaf(-ch, h, sh * c);
        ch = fmaf(sh, h, ch * c);
        sh = sh1;
    } else {
        sincos_near0(0.5f * dE, &sh, &ch);
    }
    float sn = 2.0f * sh * ch, omc = 2.0f * sh * sh;
    float dC = -r.cE * omc - r.sE * sn;
    float dS = r.cE * sn - r.sE * omc;
    float U = r.Uc * dC - r.Us * dS;
    float V = r.Vtr + (r.Vs * dC + r.Vc * dS);
    if (V <= 0.0f) return PT_ZBEHIND;
    float Vi = V * r.cosi;
    return FAST ? sqrt_a(fmaf(U, U, Vi * Vi)) : sqrtf(fmaf(U, U, Vi * Vi));
}


// ---------------------------------------------------------------------------
// Bulirsch's general complete elliptic integral (Bulirsch 1969, Numer. Math.
// 13, 305),
//   cel(kc, p, a, b) = int_0^{pi/2} (a cos^2 + b sin^2) /
//                      ((cos^2 + p sin^2) sqrt(cos^2 + kc^2 sin^2)) dth,
// evaluated for two (p, a, b) triples that share kc: the Gauss/Landen
// sequence of (kc, m) does not depend on (p, a, b), so the two integrals
// share its square roots.  The first triple has p = 1 (the K/E combination
// a K + (b - a) ... is folded into (a, b) by the caller), the second has
// p = rho > 0 and b = 0.  Converged when the arithmetic-geometric means agree
// to 3e-4 (quadratic convergence then leaves ~1e-7); at most 10 steps.
// The two integrals' updates run as the two lanes of fma/mul/add.rn.f32x2
// (one instruction for both; each lane rounded as the scalar operation).
// ---------------------------------------------------------------------------
// two-lane FP32 helpers (sm_100 and later); each lane is one IEEE operation
// rounded once, the same result as the scalar instruction
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi)
{
    return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float f2_lo(unsigned long long v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float f2_hi(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ void cel2(float kc, float a1, float b1, float srho, float a2, float *r1,
                                     float *r2)
{
    // lanes: (first integral, second integral); srho = sqrt(rho).  The lanes'
    // p start at 1 and sqrt(rho) >= 1 and only grow, kc in (0, 1] and e = kc m
    // stay normal numbers, so the .ftz approximations never meet a denormal.
    unsigned long long A = f2_pack(a1, a2), B = f2_pack(b1, 0.0f), P = f2_pack(1.0f, srho);
    float m = 1.0f, e = kc;
#pragma unroll 1
    for (int it = 0; it < 10; ++it) {
        const unsigned long long ip = f2_pack(rcp_a(f2_lo(P)), rcp_a(f2_hi(P)));
        const unsigned long long F = A;
        A = f2_fma(B, ip, A);
        const unsigned long long G = f2_mul(f2_pack(e, e), ip);
        B = f2_fma(F, G, B);
        B = f2_add(B, B);
        P = f2_add(P, G);
        float g = m;
        m = kc + m;
        if (fabsf(g - kc) <= g * 3e-4f) break;
        kc = 2.0f * sqrt_a(e);
        e = kc * m;
    }
    *r1 = (0.5f * PT_PI_F) * fmaf(f2_lo(A), m, f2_lo(B)) * rcp_a(m * (m + f2_lo(P)));
    *r2 = (0.5f * PT_PI_F) * fmaf(f2_hi(A), m, f2_hi(B)) * rcp_a(m * (m + f2_hi(P)));
}

// cel2's loop carrying K = cel(kc, 1, 1, 1) and E = cel(kc, 1, 1, kc^2) in place
// of one combination of them (cel with p = 1 is linear in (a, b), so
// cel(kc, 1, cK + cE, cK + cE kc^2) = cK K + cE E), for callers that also need
// K and E themselves.
__device__ __forceinline__ void cel3(float kc, float srho, float a2, float *K, float *E, float *r2)
{
    float p1 = 1.0f;
    float p2 = srho;   // argument ranges as in cel2
    float aK = 1.0f, bK = 1.0f, aE = 1.0f, bE = kc * kc, b2 = 0.0f;
    float m = 1.0f, e = kc;
#pragma unroll 1
    for (int it = 0; it < 10; ++it) {
        float ip1 = rcp_a(p1);
        float ip2 = rcp_a(p2);
        float g = e * ip1;
        float f = aK;
        aK = fmaf(bK, ip1, aK);
        bK = 2.0f * fmaf(f, g, bK);
        f = aE;
        aE = fmaf(bE, ip1, aE);
        bE = 2.0f * fmaf(f, g, bE);
        p1 += g;
        f = a2;
        a2 = fmaf(b2, ip2, a2);
        g = e * ip2;
        b2 = 2.0f * fmaf(f, g, b2);
        p2 += g;
        g = m;
        m = kc + m;
        if (fabsf(g - kc) <= g * 3e-4f) break;
        kc = 2.0f * sqrt_a(e);
        e = kc * m;
    }
    const float den = (0.5f * PT_PI_F) * rcp_a(m * (m + p1));
    *K = fmaf(aK, m, bK) * den;
    *E = fmaf(aE, m, bE) * den;
    *r2 = (0.5f * PT_PI_F) * fmaf(a2, m, b2) * rcp_a(m * (m + p2));
}

// ---------------------------------------------------------------------------
// Mandel & Agol (2002) terms for the quadratic law, FP32.
//   le = lambda_e, ld = lambda_d + 2/3 Theta(p - z), ed = eta_d.
//
// Geometry: d = z + p - 1, 1 - a = (1 - z + p)(1 + z - p), b - 1 = d (1 + z + p),
// q = (p - z)(p + z); all formed from single differences so they keep
// relative precision at the contact points.  kap0, kap1 and the triangle
// area come from atan2 of the Heron area (no acos of a rounded cosine).
//
// lambda_1 (partial) and lambda_2 (inside) are Mandel & Agol's
//   pref {cK K(k) + cE E(k) + cP Pi(n, k)}.
// Near z = 1 - p the modulus tends to 1 and K, Pi diverge logarithmically
// while their divergences cancel.  The kernel removes the cancellation
// algebraically:  with rho = 1 - n,
//   cP Pi = (cP/rho) K + cP (rho - 1)/rho * cel(kc, rho, 1, 0),
// and cK' = cK + cP/rho factors through b - 1:
//   lambda_1: cK' = -(b-1)(6 p^2 + 2 p z - 3),              cR = -3 q (1-a)/a
//   lambda_2: cK' = (b-1)(p^3 - p^2 z - p z^2 + 2p + z^3 - 4z)/(p+z),
//             cR = -12 q z p / (a b)
// so the brace is cel(kc, 1, cK'+cE, cK'+cE kc^2) + cel(kc, rho, cR, 0), two
// bounded integrals evaluated in one shared loop (cel2).  With a = (z-p)^2,
// b = (z+p)^2 and q = -(z-p)(z+p) these reduce exactly to
//   lambda_1: sqrt(rho) = 1/|z-p|,        cR = 3 (z+p)(1-a)/(z-p),
//   lambda_2: sqrt(rho) = (z+p)/|z-p|,    cR = 12 z p / ((z-p)(z+p)),
// which the kernel evaluates (fewer roundings; z = p is a separate case).
// Reciprocals and square roots are the one-instruction approximations.  For
// p >= 1e-15 every argument they get is a normal number or zero: d and z - p
// are 0 (separate cases) or at least an ulp of p, z or 1, and the products
// formed from them stay far above 2^-126.
// Exact special cases of Mandel & Agol's Table 1 that the general formulas
// cannot evaluate (z = 1 - p, z = p, p = z = 1/2, star covered) are taken
// separately; near them the general formulas stay accurate in FP32.
// ---------------------------------------------------------------------------
// With KE, K and E of the general cases' modulus (cases 2, 3, 8, 9: the
// partial and inside overlaps) come back too, *have_ke = true; other cases
// leave *have_ke false.
template <bool KE = false>
__device__ __forceinline__ void ma_terms(float p, float z, float *le, float *ld, float *ed, float *Kout = nullptr,
                                         float *Eout = nullptr, bool *have_ke = nullptr)
{
    if (KE) *have_ke = false;
    *le = 0.0f;
    *ld = 0.0f;
    *ed = 0.0f;
    if (!(z < 1.0f + p) || !(p > 0.0f)) return;    // out of transit (also PT_ZBEHIND, NaN)
    if (p >= 1.0f && z <= p - 1.0f) {               // case 11: star covered
        *le = 1.0f;
        *ld = 2.0f / 3.0f;
        *ed = 0.5f;
        return;
    }
    const float pi = PT_PI_F;
    float p2 = p * p, z2 = z * z;
    float d = (z - 1.0f) + p;
    float oma = (1.0f - z + p) * (1.0f + z - p);
    float bm1 = d * (1.0f + z + p);
    float zmp = z - p;
    float eta2 = 0.5f * p2 * (p2 + 2.0f * z2);
    bool inside = d < 0.0f;

    // lens geometry: only the partial (and contact) cases need it
    float le_part = p2, eta1 = eta2;
    if (!inside) {
        float fa = sqrt_a(oma * bm1);                    // 4 x triangle area (oma, bm1 >= 0)
        float k1 = atan2_pos(fa, 1.0f - p2 + z2);
        float k0 = atan2_pos(fa, p2 + z2 - 1.0f);
        le_part = (p2 * k0 + k1 - 0.5f * fa) * (1.0f / pi);
        eta1 = (k1 + 2.0f * eta2 * k0 - 0.25f * (1.0f + 5.0f * p2 + z2) * fa) * (0.5f / pi);
    }

    // parameters of the shared elliptic evaluation
    float kc, cKp, cE, srho = 1.0f, cR = 0.0f, pref, cst = 0.0f;
    bool need_cel = true;
    float e_out = inside ? eta2 : eta1;
    if (d == 0.0f) {                                 // case 4: lambda_5, z = 1 - p
        cst = 2.0f / (3.0f * pi) * acosf(1.0f - 2.0f * p) -
              4.0f / (9.0f * pi) * (3.0f + 2.0f * p - 8.0f * p2) * sqrtf(p * (1.0f - p)) -
              (p > 0.5f ? 2.0f / 3.0f : 0.0f);
        e_out = eta2;
        need_cel = false;
        kc = 1.0f; cKp = 0.0f; cE = 0.0f; pref = 0.0f;
    } else if (zmp == 0.0f) {                        // z = p
        if (p == 0.5f) {                             // case 6
            cst = 1.0f / 3.0f - 4.0f / (9.0f * pi);
            e_out = 3.0f / 32.0f;
            need_cel = false;
            kc = 1.0f; cKp = 0.0f; cE = 0.0f; pref = 0.0f;
        } else if (p < 0.5f) {                       // case 5: lambda_4, modulus 2p
            kc = sqrtf((1.0f - 2.0f * p) * (1.0f + 2.0f * p));
            cKp = 1.0f - 4.0f * p2;
            cE = 4.0f * (2.0f * p2 - 1.0f);
            pref = 2.0f / (9.0f * pi);
            cst = 1.0f / 3.0f;
            e_out = eta2;
        } else {                                     // case 7: lambda_3, modulus 1/(2p)
            kc = sqrtf((2.0f * p - 1.0f) * (2.0f * p + 1.0f)) / (2.0f * p);
            cKp = -(1.0f - 4.0f * p2) * (3.0f - 8.0f * p2) / p;
            cE = 16.0f * p * (2.0f * p2 - 1.0f);
            pref = 1.0f / (9.0f * pi);
            cst = 1.0f / 3.0f;
            e_out = eta1;
        }
    } else if (inside) {                             // cases 3, 9: lambda_2
        kc = sqrt_a(-bm1 * rcp_a(oma));
        cKp = bm1 * (p2 * p - p2 * z - p * z2 + 2.0f * p + z2 * z - 4.0f * z) * rcp_a(p + z);
        cE = oma * (z2 + 7.0f * p2 - 4.0f);
        srho = (p + z) * rcp_a(fabsf(zmp));
        cR = (12.0f * z * p) * rcp_a(zmp * (z + p));
        pref = 2.0f * rcp_a(9.0f * pi * sqrt_a(oma));
    } else {                                         // cases 2, 8: lambda_1
        kc = sqrt_a(bm1 * rcp_a(4.0f * z * p));
        cKp = -bm1 * (6.0f * p2 + 2.0f * p * z - 3.0f);
        cE = 4.0f * p * z * (z2 + 7.0f * p2 - 4.0f);
        srho = rcp_a(fabsf(zmp));
        cR = (3.0f * (p + z) * oma) * rcp_a(zmp);
        pref = rcp_a(9.0f * pi * sqrt_a(p * z));
    }
    float lam = cst;
    if (need_cel) {
        float r1, r2;
        if (KE && d != 0.0f && zmp != 0.0f) {
            float K, E;
            cel3(kc, srho, cR, &K, &E, &r2);
            r1 = fmaf(cKp, K, cE * E);
            *Kout = K;
            *Eout = E;
            *have_ke = true;
        } else {
            cel2(kc, cKp + cE, fmaf(cE, kc * kc, cKp), srho, cR, &r1, &r2);
        }
        lam = fmaf(pref, r1 + r2, cst);
    }
    if (p > z) lam += 2.0f / 3.0f;
    *le = inside ? p2 : le_part;
    *ld = lam;
    *ed = e_out;
}

// Bilinear interpolation of the tabulated Mandel-Agol terms (Sec. 2.2.3):
// node (i, j) holds the terms at k_i = k_lo + i dk, z_j = j dz with
// dz = (1 + k_hi) / (n_z - 1).  Out of transit (z >= 1 + k, also the
// behind-the-star sentinel and NaN) the terms are zero; k is clamped to the
// table's range.
__device__ __forceinline__ void ma_interp(const float4 *tab, int n_k, int n_z, float k_lo, float k_hi,
                                          float inv_dk, float inv_dz, float k, float z, float *le, float *ld,
                                          float *ed)
{
    *le = 0.0f;
    *ld = 0.0f;
    *ed = 0.0f;
    if (!(z < 1.0f + k)) return;
    float fk = (fminf(fmaxf(k, k_lo), k_hi) - k_lo) * inv_dk;
    int ik = min((int)fk, n_k - 2);
    float wk = fk - (float)ik;
    float fz = fminf(fmaxf(z, 0.0f) * inv_dz, (float)(n_z - 1));
    int iz = min((int)fz, n_z - 2);
    float wz = fz - (float)iz;
    const float4 *r0 = tab + (size_t)ik * n_z + iz;
    const float4 *r1 = r0 + n_z;
    float4 a = __ldg(r0), b = __ldg(r0 + 1), c = __ldg(r1), d = __ldg(r1 + 1);
    float a0 = fmaf(wz, b.x - a.x, a.x), a1 = fmaf(wz, b.y - a.y, a.y), a2 = fmaf(wz, b.z - a.z, a.z);
    float c0 = fmaf(wz, d.x - c.x, c.x), c1 = fmaf(wz, d.y - c.y, c.y), c2 = fmaf(wz, d.z - c.z, c.z);
    *le = fmaf(wk, c0 - a0, a0);
    *ld = fmaf(wk, c1 - a1, a1);
    *ed = fmaf(wk, c2 - a2, a2);
}

// Network coordinate across the ingress/egress band: theta = acos(1 - 2 s)
// mapped to [-1, 1].  Near both contacts (s -> 0, s -> 1) the MA terms
// behave like powers of sqrt(s) and sqrt(1 - s); in theta they are regular.
__device__ __forceinline__ float band_coord(float s)
{
    return acosf(fminf(1.0f, fmaxf(-1.0f, 1.0f - 2.0f * s))) * (2.0f / PT_PI_F) - 1.0f;
}

// lambda_e alone (the lens area over pi), for callers that take lambda_d and
// eta_d from elsewhere: the same geometry as ma_terms.
__device__ __forceinline__ float lens_le(float p, float z)
{
    if (!(z < 1.0f + p) || !(p > 0.0f)) return 0.0f;
    if (p >= 1.0f && z <= p - 1.0f) return 1.0f;
    float d = (z - 1.0f) + p;
    if (d <= 0.0f) return p * p;
    float p2 = p * p, z2 = z * z;
    float oma = (1.0f - z + p) * (1.0f + z - p);
    float fa = sqrtf(fmaxf(0.0f, oma * d * (1.0f + z + p)));
    float k1 = atan2f(fa, 1.0f - p2 + z2);
    float k0 = atan2f(fa, p2 + z2 - 1.0f);
    return (p2 * k0 + k1 - 0.5f * fa) * (1.0f / PT_PI_F);
}

// Quadratic-law weights of Eq. (ma_model): f = 1 - (we le + wd ld + wn ed),
// with c = u1 + 2 u2 and the normalisation 1 - u1/3 - u2/6.
__device__ __forceinline__ void ma_weights(float u1, float u2, float *we, float *wd, float *wn)
{
    float inv = 1.0f / (1.0f - u1 * (1.0f / 3.0f) - u2 * (1.0f / 6.0f));
    float c = u1 + 2.0f * u2;
    *we = (1.0f - c) * inv;
    *wd = c * inv;
    *wn = u2 * inv;
}

constexpr double PT_PI_D = 3.14159265358979323846;

__device__ __forceinline__ float wrap_pos(float x)   // into [0, 2 pi); closed form, no loop
{
    const float tp = 6.28318530717958f;
    float y = x - tp * floorf(x / tp);
    return (y >= tp) ? 0.0f : y;
}

__device__ __forceinline__ float wrap_neg(float x)   // into (-2 pi, 0]
{
    const float tp = 6.28318530717958f;
    float y = wrap_pos(x);
    return (y > 0.0f) ? y - tp : 0.0f;
}

// Per-geometry record (see GeomRec): double-float t0/P, the conjunction
// anchor of an eccentric orbit (FP64 here; it enters the hot path only as
// coefficients of small terms), sky-plane position coefficients, and a
// conservative transit window in time for radius ratio k, widened by half
// an exposure.
__device__ __forceinline__ void make_geom_rec(double t0, double P, float a_f, float inc, bool ecc, float e_f,
                                              float w_f, float k, float half_exp, GeomRec *out)
{
    GeomRec r;
    r.t0h = (float)t0;
    r.t0l = (float)(t0 - (double)r.t0h);
    r.Ph = (float)P;
    r.Pl = (float)(P - (double)r.Ph);
    r.invP = (float)(1.0 / P);
    r.nang = (float)(2.0 * PT_PI_D / P);
    double a = a_f;
    double ci = cos((double)inc);
    r.a = (float)a;
    r.cosi = (float)ci;
    r.k = k;
    double e = 0.0, w = 0.5 * PT_PI_D;
    if (ecc) {
        e = e_f;
        w = w_f;
    }
    r.ecc = ecc ? 1.0f : 0.0f;
    // conjunction anchor: f_tr = pi/2 - w, E_tr from tan(E/2) = sqrt((1-e)/(1+e)) tan(f/2).
    // FP32 suffices: the anchor's sine and cosine only scale the small
    // differential terms of orbit_z (relative error ~1e-7 there), and the
    // sky position at conjunction is zero by construction, not computed.
    float ef = (float)e, wf = (float)w;
    float ftrf = 0.5f * PT_PI_F - wf;
    float Etrf = 2.0f * atan2f(sqrtf(1.0f - ef) * sinf(0.5f * ftrf), sqrtf(1.0f + ef) * cosf(0.5f * ftrf));
    float sEf, cEf, swf, cwf;
    sincosf(Etrf, &sEf, &cEf);
    sincosf(wf, &swf, &cwf);
    float sef = sqrtf((1.0f - ef) * (1.0f + ef)), af = (float)a;
    double ftr = 0.5 * PT_PI_D - w;
    double Etr = Etrf, sE = sEf;
    r.ecE = ef * cEf;
    r.esE = ef * sEf;
    r.cE = cEf;
    r.sE = sEf;
    r.Uc = af * cwf;
    r.Us = af * sef * swf;
    r.Vs = af * swf;
    r.Vc = af * sef * cwf;
    r.Vtr = af * (1.0f - ef * cEf);
    r.nq = ecc ? (float)(e / (1.0 - e)) : 0.0f;
    r.pad1 = r.pad2 = 0.0f;
    // Conservative window.  z^2 >= r_min^2 (sin^2(th) sin^2 i + cos^2 i) with
    // th = w + f - pi/2 and r_min = a (1 - e), so z > 1 + k whenever
    // sin^2 th > ((1+k)^2 / r_min^2 - cos^2 i) / sin^2 i.  The true-anomaly
    // window [f_tr - th_w, f_tr + th_w] maps to a mean-anomaly window and
    // from there to time; widened by half an exposure and a margin.
    float rr = (1.0f + fabsf(k)) * 1.0001f + 1e-5f;
    float rmin = (float)(a * (1.0 - e));
    float ci2 = (float)(ci * ci), si2 = 1.0f - ci2;
    float lo, hi;
    float full = 1.5f * (float)P;
    if (rmin * (float)fabs(ci) >= rr) {
        lo = 1.0f;
        hi = -1.0f;   // never in transit
    } else {
        float s2 = (rr * rr / (rmin * rmin) - ci2) / fmaxf(si2, 1e-30f);
        if (s2 >= 1.0f) {
            lo = -full;
            hi = full;
        } else {
            float thw = asinf(sqrtf(fmaxf(s2, 0.0f))) * 1.001f + 1e-5f;
            if (ecc && e > 0.0) {
                // r = a (1 - e^2) / (1 + e cos f) is smallest where cos f is
                // largest; over f in [f_tr - thw, f_tr + thw] that bound is
                // much tighter than a (1 - e), and the window it gives
                // (narrower, so the bound still holds on it) is conservative.
                float ftr_f = (float)ftr;
                float f1 = ftr_f - thw, f2 = ftr_f + thw;
                float cmax = fmaxf(cosf(f1), cosf(f2));
                float f0 = 6.28318530717958f * ceilf(f1 / 6.28318530717958f);   // first multiple of 2 pi >= f1
                if (f0 <= f2) cmax = 1.0f;
                float ef2 = (float)e;
                float rmin2 = (float)a * (1.0f - ef2 * ef2) / (1.0f + ef2 * cmax) * 0.9999f;
                float s2b = (rr * rr / (rmin2 * rmin2) - ci2) / fmaxf(si2, 1e-30f);
                if (rmin2 > rmin && s2b < s2) thw = asinf(sqrtf(fmaxf(s2b, 0.0f))) * 1.001f + 1e-5f;
            }
            float margin = half_exp + 1e-6f + 1e-6f * (float)P;
            if (!ecc) {
                lo = -thw / r.nang - margin;
                hi = thw / r.nang + margin;
            } else {
                float ef = (float)e, ftrf = (float)ftr;
                float se2 = sqrtf(1.0f - ef), se1 = sqrtf(1.0f + ef);
                float El = 2.0f * atan2f(se2 * sinf(0.5f * (ftrf - thw)), se1 * cosf(0.5f * (ftrf - thw)));
                float Eh = 2.0f * atan2f(se2 * sinf(0.5f * (ftrf + thw)), se1 * cosf(0.5f * (ftrf + thw)));
                float Mtr = (float)(Etr - e * sE);
                float Ml = wrap_neg(El - ef * sinf(El) - Mtr);
                float Mh = wrap_pos(Eh - ef * sinf(Eh) - Mtr);
                if (Mh - Ml >= 3.0f) {
                    lo = -full;
                    hi = full;
                } else {
                    lo = Ml * 1.0005f / r.nang - margin;
                    hi = Mh * 1.0005f / r.nang + margin;
                }
            }
        }
    }
    r.win_lo = lo;
    r.win_hi = hi;
    *out = r;
}


// Warp-aggregated append to a shared-memory queue; returns the slot.
__device__ __forceinline__ int warp_append(int *counter, bool pred)
{
    unsigned mask = __ballot_sync(0xffffffffu, pred);
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (mask != 0u && lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader < 0 ? 0 : leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

}  // namespace pt
