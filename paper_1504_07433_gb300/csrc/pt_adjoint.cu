// pt_adjoint.cu -- hand-written adjoint of the quadratic Mandel-Agol light
// curve: SSR = sum_t wt (y - f)^2 and dSSR/dtheta for
// theta = (t0, P, a, b, e, w, k, u1, u2), one CTA per parameter vector, the
// forward model recomputed in registers (nothing saved between passes).
//
// The paper has no gradients (it cites analytic MA derivatives, Pal 2008).
// They follow from the definition of the occulted flux: with
// I_g = int int_overlap g dA for g in {1, mu, mu^2},
//   F = 1 - [(1 - u1 - u2) I_1 + (u1 + 2 u2) I_mu - u2 I_mu2] / (pi (1 - u1/3 - u2/6)),
// and only the planet's edge inside the star moves with k or z, so
//   dI_g/dk = k int_arc g dphi,   dI_g/dz = k int_arc g cos(phi) dphi,
// complete elliptic integrals for g = mu.  The orbit part is the chain rule
// through z = sqrt(U^2 + V^2 cos^2 i), Kepler's equation (solved in the same
// differential FP32 form as the forward kernels) and the conjunction anchor.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../../include/pt.h"
#include "pt_device.cuh"

namespace pt_internal {
int set_error(int status, const char *where, const char *msg);   // pt_lc.cu
}

namespace {

constexpr int TB = 128;
constexpr float PI_F = 3.14159265358979f;

// cel(kc, 1, a, b) for two (a, b) pairs sharing kc and p = 1 (so the whole
// Landen sequence, including p, is shared): returns K and E.
__device__ __forceinline__ void ellke(float kc, float *K, float *E)
{
    float a1 = 1.0f, b1 = 1.0f;          // K
    float a2 = 1.0f, b2 = kc * kc;       // E
    float p = 1.0f, m = 1.0f, e = kc;
#pragma unroll 1
    for (int it = 0; it < 10; ++it) {
        float ip = pt::rcp_a(p);   // p, kc, e, m normal throughout (as in pt::cel2)
        float g = e * ip;
        float f = a1;
        a1 = fmaf(b1, ip, a1);
        b1 = 2.0f * fmaf(f, g, b1);
        f = a2;
        a2 = fmaf(b2, ip, a2);
        b2 = 2.0f * fmaf(f, g, b2);
        p += g;
        g = m;
        m = kc + m;
        if (fabsf(g - kc) <= g * 3e-4f) break;
        kc = 2.0f * pt::sqrt_a(e);
        e = kc * m;
    }
    float den = pt::rcp_a(m * (m + p));
    *K = (0.5f * PI_F) * fmaf(a1, m, b1) * den;
    *E = (0.5f * PI_F) * fmaf(a2, m, b2) * den;
}

// S(m) = int_0^{pi/2} sin^2 cos^2 / sqrt(1 - m sin^2): binomial series below
// m = 1/2 (terms fall as m^n n^-2; 24 terms reach 1e-9), closed form in K, E
// at and above it.  Term n is c_n (w_n - w_{n+1}) m^n with c_n the binomial
// coefficients of (1 - x)^(-1/2) and w_n = int_0^{pi/2} sin^(2n) = (pi/2)
// (2n-1)!!/(2n)!!; the coefficients are constants, formed at compile time,
// and the sum runs by Horner's rule.
struct S2C2Coef {
    float a[24];
};

constexpr S2C2Coef make_s2c2()
{
    S2C2Coef r{};
    double c = 1.0, w1 = 0.25 * 3.14159265358979323846, w2 = w1 * 0.75;
    for (int n = 0; n < 24; ++n) {
        r.a[n] = (float)(c * (w1 - w2));
        c *= (2.0 * n + 1.0) / (2.0 * n + 2.0);
        double w3 = w2 * (2.0 * n + 5.0) / (2.0 * n + 6.0);
        w1 = w2;
        w2 = w3;
    }
    return r;
}

__device__ __forceinline__ float s2c2_int(float m, float K, float E)
{
    if (m < 0.5f) {
        constexpr S2C2Coef C = make_s2c2();
        float s = C.a[23];
#pragma unroll
        for (int n = 22; n >= 0; --n) s = fmaf(s, m, C.a[n]);
        return s;
    }
    return ((2.0f - m) * E - 2.0f * (1.0f - m) * K) * pt::rcp_a(3.0f * m * m);   // m >= 1/2
}

// Overlap integrals I (x pi-free form: I_1 = pi le, I_mu = pi ld', I_mu2 =
// pi (le - ed)) and their derivatives d[0..5] = dI_1/dk, dI_1/dz, dI_mu/dk,
// dI_mu/dz, dI_mu2/dk, dI_mu2/dz.
__device__ __forceinline__ void overlap_derivs(float p, float z, float *d, bool have_ke = false, float Kin = 0.0f,
                                               float Ein = 0.0f)
{
    for (int i = 0; i < 6; ++i) d[i] = 0.0f;
    if (!(z < 1.0f + p) || !(p > 0.0f)) return;
    if (p >= 1.0f && z <= p - 1.0f) return;
    float oma = (1.0f - z + p) * (1.0f + z - p);
    float dd = (z - 1.0f) + p;
    float al = 1.0f - z * z - p * p;
    if (dd < 0.0f) {                                   // full circle inside the star
        // oma, -dd and z p are normal numbers here (as in pt::ma_terms)
        const float ioma = pt::rcp_a(oma);
        float m = 4.0f * z * p * ioma;
        float K = Kin, E = Ein;
        if (!have_ke) ellke(pt::sqrt_a(-dd * (1.0f + z + p) * ioma), &K, &E);
        float so = pt::sqrt_a(oma);
        d[0] = 2.0f * PI_F * p;
        d[2] = 4.0f * p * so * E;
        d[3] = -p * 4.0f * so * m * s2c2_int(m, K, E);
        d[4] = p * al * 2.0f * PI_F;
        d[5] = -p * 2.0f * z * p * PI_F;
        return;
    }
    float bm1 = dd * (1.0f + z + p);
    float fa = pt::sqrt_a(fmaxf(0.0f, oma * bm1));
    float kap0 = pt::atan2_pos(fa, p * p + z * z - 1.0f);
    float ipz = pt::rcp_a(2.0f * p * z);
    float sk = fa * ipz, ck = (p * p + z * z - 1.0f) * ipz;
    float m1 = 0.5f * oma * ipz, mc1 = 0.5f * bm1 * ipz;
    const float szp = pt::sqrt_a(z * p);
    float K, E, mcK;
    if (dd == 0.0f) {                                  // contact with the limb from inside: m1 = 1
        E = 1.0f;
        mcK = 0.0f;
    } else {
        if (have_ke) {
            K = Kin;
            E = Ein;
        } else {
            ellke(pt::sqrt_a(mc1), &K, &E);
        }
        mcK = mc1 * K;
    }
    float icos = -2.0f * sk, icos2 = kap0 + sk * ck;
    d[0] = 2.0f * p * kap0;
    d[1] = p * icos;
    d[2] = 8.0f * p * szp * (E - mcK);
    d[3] = -p * (8.0f / 3.0f) * szp * ((2.0f * m1 - 1.0f) * E + mcK);
    d[4] = p * (al * 2.0f * kap0 - 2.0f * z * p * icos);
    d[5] = p * (al * icos - 2.0f * z * p * icos2);
}

struct VecConst {
    pt::GeomRec g;          // phase reduction, window, anchor, position coefficients
    float e, w, se, sw, cw, b;
    float ci, dci_a, dci_b, dci_e, dci_w;
    float dMtr_de, dMtr_dw;
    float k, u1, u2, c0, c2, D;
    float invPD, inv3D, inv6D, ise;   // 1 / (pi D), 1 / (3 D), 1 / (6 D), 1 / se
};

__device__ void make_const(const pt_theta &th, int v, float half_exp, VecConst *c)
{
    const float PI2 = 6.28318530717958f;
    double t0 = th.t0[v], P = th.P[v];
    pt::GeomRec &r = c->g;
    r.t0h = (float)t0;
    r.t0l = (float)(t0 - (double)r.t0h);
    r.Ph = (float)P;
    r.Pl = (float)(P - (double)r.Ph);
    r.invP = (float)(1.0 / P);
    r.nang = (float)(2.0 * 3.14159265358979323846 / P);
    float a = th.a[v], b = th.b[v], e = th.e ? th.e[v] : 0.0f, w = th.w ? th.w[v] : 0.5f * PI_F;
    float k = th.k[v];
    float sw, cw;
    sincosf(w, &sw, &cw);
    float se = sqrtf((1.0f - e) * (1.0f + e));
    float ome2 = (1.0f - e) * (1.0f + e);
    float ci = b * (1.0f + e * sw) / (a * ome2);
    c->e = e;
    c->w = w;
    c->se = se;
    c->sw = sw;
    c->cw = cw;
    c->b = b;
    c->ci = ci;
    c->dci_a = -ci / a;
    c->dci_b = (1.0f + e * sw) / (a * ome2);
    c->dci_e = b / a * (sw * ome2 + 2.0f * e * (1.0f + e * sw)) / (ome2 * ome2);
    c->dci_w = b / a * e * cw / ome2;
    // conjunction anchor (FP32: it enters only as coefficients of small terms)
    float ftr = 0.5f * PI_F - w;
    float Etr = 2.0f * atan2f(sqrtf(1.0f - e) * sinf(0.5f * ftr), sqrtf(1.0f + e) * cosf(0.5f * ftr));
    float sE, cE;
    sincosf(Etr, &sE, &cE);
    float ecEt = 1.0f - e * cE;
    c->dMtr_dw = -ecEt * ecEt / se;
    c->dMtr_de = -ecEt * sE / ome2 - sE;
    r.a = a;
    r.cosi = ci;
    r.k = k;
    r.ecc = 1.0f;
    r.ecE = e * cE;
    r.esE = e * sE;
    r.cE = cE;
    r.sE = sE;
    r.Uc = a * cw;
    r.Us = a * se * sw;
    r.Vs = a * sw;
    r.Vc = a * se * cw;
    r.Vtr = a * ecEt;
    // conservative window (as the forward set-up): |sin th| > sqrt(((1+k)^2/rmin^2 - ci^2)/(1 - ci^2))
    float rr = (1.0f + k) * 1.0001f + 1e-5f;
    float rmin = a * (1.0f - e);
    float ci2 = ci * ci;
    float lo, hi, full = 1.5f * (float)P;
    if (rmin * fabsf(ci) >= rr) {
        lo = 1.0f;
        hi = -1.0f;
    } else {
        float s2 = (rr * rr / (rmin * rmin) - ci2) / fmaxf(1.0f - ci2, 1e-30f);
        if (s2 >= 1.0f) {
            lo = -full;
            hi = full;
        } else {
            float thw = asinf(sqrtf(fmaxf(s2, 0.0f))) * 1.001f + 1e-5f;
            float margin = half_exp + 1e-6f + 1e-6f * (float)P;
            float s1e = sqrtf(1.0f - e), s1p = sqrtf(1.0f + e);
            float El = 2.0f * atan2f(s1e * sinf(0.5f * (ftr - thw)), s1p * cosf(0.5f * (ftr - thw)));
            float Eh = 2.0f * atan2f(s1e * sinf(0.5f * (ftr + thw)), s1p * cosf(0.5f * (ftr + thw)));
            float Mtr = Etr - e * sE;
            float Ml = El - e * sinf(El) - Mtr;
            Ml = Ml - PI2 * floorf(Ml / PI2);
            Ml = (Ml > 0.0f) ? Ml - PI2 : 0.0f;
            float Mh = Eh - e * sinf(Eh) - Mtr;
            Mh = Mh - PI2 * floorf(Mh / PI2);
            if (Mh >= PI2) Mh = 0.0f;
            if (Mh - Ml >= 3.0f) {
                lo = -full;
                hi = full;
            } else {
                lo = Ml * 1.0005f / r.nang - margin;
                hi = Mh * 1.0005f / r.nang + margin;
            }
        }
    }
    r.win_lo = lo;
    r.win_hi = hi;
    r.nq = (float)(e / (1.0 - e));
    r.pad1 = r.pad2 = 0.0f;
    c->k = k;
    c->u1 = th.u1[v];
    c->u2 = th.u2[v];
    c->c0 = 1.0f - c->u1 - c->u2;
    c->c2 = c->u1 + 2.0f * c->u2;
    c->D = 1.0f - c->u1 * (1.0f / 3.0f) - c->u2 * (1.0f / 6.0f);
    c->invPD = 1.0f / (PI_F * c->D);
    c->inv3D = 1.0f / (3.0f * c->D);
    c->inv6D = 1.0f / (6.0f * c->D);
    c->ise = 1.0f / c->se;
}

// Flux and its gradient at one (time, supersample) point.
__device__ __forceinline__ float point_grad(const VecConst &c, float dts, float n_ep, int max_iter, bool *bad,
                                            float *g)
{
    const pt::GeomRec &r = c.g;
    float dM = r.nang * dts;
    float dE = dM / (1.0f - r.ecE);
    float sh, ch;
    bool conv = false;
    for (int it = 0; it < max_iter; ++it) {
        pt::sincos_near0(0.5f * dE, &sh, &ch);
        float sn = 2.0f * sh * ch, omc = 2.0f * sh * sh;
        float F = (dE - r.ecE * sn) + (r.esE * omc - dM);
        float Fp = 1.0f - r.ecE * (1.0f - omc) + r.esE * sn;
        float step = F * pt::rcp_a(Fp);   // Fp lies in [1 - e, 1 + e]
        dE -= step;
        if (fabsf(step) <= 4e-7f * fabsf(dE) + 1e-12f) {
            conv = true;
            break;
        }
    }
    if (!conv) *bad = true;
    pt::sincos_near0(0.5f * dE, &sh, &ch);
    float sn = 2.0f * sh * ch, omc = 2.0f * sh * sh;
    float dC = -r.cE * omc - r.sE * sn;
    float dS = r.cE * sn - r.sE * omc;
    float U = r.Uc * dC - r.Us * dS;
    float V = r.Vtr + (r.Vs * dC + r.Vc * dS);
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = 0.0f;
    if (V <= 0.0f) return 1.0f;
    float Vi = V * c.ci;
    float z = sqrtf(fmaf(U, U, Vi * Vi));
    float le, ld, ed, Kc = 0.0f, Ec = 0.0f;
    bool have_ke = false;
    pt::ma_terms<true>(c.k, z, &le, &ld, &ed, &Kc, &Ec, &have_ke);
    if (le == 0.0f && ld == 0.0f && ed == 0.0f) return 1.0f;
    const float pi = PI_F;
    float I0 = pi * le, I1 = pi * ld, I2 = pi * (le - ed);
    float N = c.c0 * I0 + c.c2 * I1 - c.u2 * I2;
    const float invPD = c.invPD;
    float f = 1.0f - N * invPD;
    float d[6];
    overlap_derivs(c.k, z, d, have_ke, Kc, Ec);
    float dFdk = -(c.c0 * d[0] + c.c2 * d[2] - c.u2 * d[4]) * invPD;
    float dFdz = -(c.c0 * d[1] + c.c2 * d[3] - c.u2 * d[5]) * invPD;
    g[6] = dFdk;
    g[7] = -((I1 - I0) * invPD + N * invPD * c.inv3D);
    g[8] = -((2.0f * I1 - I0 - I2) * invPD + N * invPD * c.inv6D);
    // chain rule through the orbit
    float cE = r.cE + dC, sE = r.sE + dS;
    float a = r.a, e = c.e, se = c.se, sw = c.sw, cw = c.cw, ci = c.ci;
    float iecE = pt::rcp_a(1.0f - e * cE);   // in [1/(1+e), 1/(1-e)]
    float zinv = 1.0f / z;
    // i = 0 (t0), 1 (P): only M moves
    {
        float dMi[2] = {-r.nang, -r.nang * (dts * r.invP + n_ep)};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            float dEi = dMi[i] * iecE;
            float dX = -a * sE * dEi;
            float dY = a * se * cE * dEi;
            float dU = dX * cw - dY * sw;
            float dV = dX * sw + dY * cw;
            g[i] = dFdz * (U * dU + V * ci * ci * dV) * zinv;
        }
    }
    {   // i = 2 (a)
        float dX = cE - e, dY = se * sE;
        float dU = dX * cw - dY * sw;
        float dV = dX * sw + dY * cw;
        g[2] = dFdz * (U * dU + V * ci * ci * dV + V * V * ci * c.dci_a) * zinv;
    }
    g[3] = dFdz * (V * V * ci * c.dci_b) * zinv;   // b enters through cos i only
    {   // i = 4 (e)
        float dEi = (c.dMtr_de + sE) * iecE;
        float dX = -a * sE * dEi - a;
        float dY = a * se * cE * dEi - a * e * sE * c.ise;
        float dU = dX * cw - dY * sw;
        float dV = dX * sw + dY * cw;
        g[4] = dFdz * (U * dU + V * ci * ci * dV + V * V * ci * c.dci_e) * zinv;
    }
    {   // i = 5 (w)
        float dEi = c.dMtr_dw * iecE;
        float dX = -a * sE * dEi;
        float dY = a * se * cE * dEi;
        float dU = dX * cw - dY * sw - V;
        float dV = dX * sw + dY * cw + U;
        g[5] = dFdz * (U * dU + V * ci * ci * dV + V * V * ci * c.dci_w) * zinv;
    }
    return f;
}

struct BwdArgs {
    const float2 *tsplit;
    const float2 *tile_mm;    // [n_tiles] smallest and largest time of each tile of TT times
    const double *tile_ssr;   // [n_tiles] sum of wt (y - 1)^2 over each tile
    int n_t;
    pt_theta th;
    int n_ss;
    float t_exp;
    int max_iter;
    const float *y, *wt;
    float *grad, *ssr, *flux;
    int *n_bad;
};

// Per tile of TT times (one CTA of TT threads): the double-float split of
// each time, the tile's smallest and largest time (rounded outward to FP32)
// and the residual sum of its times with the flux at 1, sum wt (y - 1)^2, in
// FP64 and a fixed order.  The adjoint kernel skips tiles that meet no
// transit window, where the flux is exactly 1 and every derivative zero, and
// takes their residual sums from here.
constexpr int TT = 64;   // times per tile

__global__ void __launch_bounds__(TT) tile_kernel(const double *t, const float *y, const float *wt, int n,
                                                  float2 *tsplit, float2 *tile_mm, double *tile_ssr)
{
    __shared__ double smin[TT / 32], smax[TT / 32], ssum[TT / 32];
    const int i = blockIdx.x * TT + threadIdx.x;
    double lo = INFINITY, hi = -INFINITY, r2 = 0.0;
    if (i < n) {
        const double x = t[i];
        const float h = (float)x;
        tsplit[i] = make_float2(h, (float)(x - (double)h));
        lo = hi = x;
        const double r = 1.0 - (double)y[i];
        r2 = (wt ? (double)wt[i] : 1.0) * r * r;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    }
    if (lane == 0) {
        smin[warp] = lo;
        smax[warp] = hi;
        ssum[warp] = r2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < TT / 32; ++w) {
            lo = fmin(lo, smin[w]);
            hi = fmax(hi, smax[w]);
            r2 += ssum[w];
        }
        float flo = (float)lo, fhi = (float)hi;
        if ((double)flo > lo) flo = nextafterf(flo, -INFINITY);
        if ((double)fhi < hi) fhi = nextafterf(fhi, INFINITY);
        tile_mm[blockIdx.x] = make_float2(flo, fhi);
        tile_ssr[blockIdx.x] = r2;
    }
}

// Can a time in [tmin, tmax] lie in the transit window of some epoch,
// t - t0 - n P in [win_lo, win_hi]?  That is, is there an integer n with
// (tmin - t0 - win_hi) / P <= n <= (tmax - t0 - win_lo) / P?  The interval
// is widened by m, 1e-6 of the magnitudes involved, which exceeds the FP32
// rounding of these expressions, so the test never misses an epoch.
__device__ __forceinline__ bool tile_meets_window(const pt::GeomRec &g, float tmin, float tmax)
{
    if (g.win_lo > g.win_hi) return false;                // never in transit
    if (g.win_hi - g.win_lo >= 0.5f * g.Ph) return true;  // a wide window: no test
    const float m = 1e-6f * (fabsf(tmin) + fabsf(tmax) + fabsf(g.t0h) + g.Ph) + 1e-9f;
    const float n_lo = ceilf((tmin - g.t0h - g.win_hi - m) * g.invP);
    const float n_hi = floorf((tmax - g.t0h - g.win_lo + m) * g.invP);
    return n_lo <= n_hi;
}


__global__ void __launch_bounds__(TB, 6) ma_bwd_kernel(BwdArgs A)
{
    __shared__ VecConst sc;
    __shared__ float sred[TB / 32][10];
    __shared__ double sout[TB / 32];
    __shared__ int slist[TB];          // the current chunk's evaluated tiles, in order
    __shared__ int swcnt[TB / 32];
    __shared__ int sbad;
    const int v = blockIdx.x;
    if (threadIdx.x == 0) {
        make_const(A.th, v, 0.5f * A.t_exp, &sc);
        sbad = 0;
    }
    __syncthreads();
    const VecConst c = sc;
    float acc[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) acc[i] = 0.0f;
    bool bad = false;
    const float inv_ss = 1.0f / (float)A.n_ss;
    const int n_tiles = (A.n_t + TT - 1) / TT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double ssr_out = 0.0;   // this thread's share of the skipped tiles' residual sums
    // Tile j holds times j TT .. j TT + TT - 1.  A tile that meets no transit
    // window has flux 1 and zero derivatives: it is skipped and its residual
    // sum comes from tile_kernel.  Chunks of TB tiles: one window test per
    // thread, the evaluated tiles listed in order in shared memory, then
    // passes over TB / TT of them at a time (thread tid takes time tid % TT of
    // list entry tid / TT), each pass's inputs loaded during the previous one.
    constexpr int TPP = TB / TT;   // tiles per pass
    for (int c0 = 0; c0 < n_tiles; c0 += TB) {
        const int jt = c0 + (int)threadIdx.x;
        bool ev = false;
        if (jt < n_tiles) {
            const float2 mm = A.tile_mm[jt];
            ev = tile_meets_window(c.g, mm.x, mm.y);
            if (!ev) ssr_out += A.tile_ssr[jt];
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ev);
        __syncthreads();   // the previous chunk's list is no longer read
        if (lane == 0) swcnt[warp] = __popc(bal);
        __syncthreads();
        int base = 0, n_ev = 0;
#pragma unroll
        for (int w = 0; w < TB / 32; ++w) {
            base += (w < warp) ? swcnt[w] : 0;
            n_ev += swcnt[w];
        }
        if (ev) slist[base + __popc(bal & ((1u << lane) - 1u))] = jt;
        if (A.flux) {
            // flux 1 on this chunk's skipped tiles: thread tid writes time
            // tid % TT of every (TB / TT)-th tile
            const int c1 = min(n_tiles, c0 + TB);
            for (int tj = c0 + (int)(threadIdx.x / TT); tj < c1; tj += TPP) {
                const int i = tj * TT + (int)(threadIdx.x % TT);
                const float2 mm = A.tile_mm[tj];
                if (i < A.n_t && !tile_meets_window(c.g, mm.x, mm.y)) A.flux[(size_t)v * A.n_t + i] = 1.0f;
            }
        }
        __syncthreads();
        // pass q takes list entries q TPP .. q TPP + TPP - 1
        auto time_of = [&](int q) {
            const int e = q * TPP + (int)(threadIdx.x / TT);
            return e < n_ev ? slist[e] * TT + (int)(threadIdx.x % TT) : -1;
        };
        const int n_pass = (n_ev + TPP - 1) / TPP;
        int i_n = n_pass > 0 ? time_of(0) : -1;
        float2 ts_n = make_float2(0.0f, 0.0f);
        float y_n = 0.0f, w_n = 1.0f;
        if (i_n >= 0 && i_n < A.n_t) {
            ts_n = A.tsplit[i_n];
            y_n = A.y[i_n];
            w_n = A.wt ? A.wt[i_n] : 1.0f;
        }
        for (int q = 0; q < n_pass; ++q) {
        const int i = i_n;
        const float2 ts = ts_n;
        const float yi = y_n, wi = w_n;
        i_n = q + 1 < n_pass ? time_of(q + 1) : -1;
        if (i_n >= 0 && i_n < A.n_t) {
            ts_n = A.tsplit[i_n];
            y_n = A.y[i_n];
            w_n = A.wt ? A.wt[i_n] : 1.0f;
        }
        if (i < 0 || i >= A.n_t) continue;
        // epoch and offset (double-float phase reduction)
        float s = ts.x - c.g.t0h;
        float n_ep = rintf(s * c.g.invP);
        float dt = 0.0f;
        bool inw = false;
        if (pt::maybe_in_window(ts.x, c.g)) {
            dt = pt::reduce_time(ts.x, ts.y, c.g);
            inw = dt >= c.g.win_lo && dt <= c.g.win_hi;
        }
        float f = 1.0f;
        float gp[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) gp[j] = 0.0f;
        if (inw) {
            f = 0.0f;
            for (int ss = 0; ss < A.n_ss; ++ss) {
                float dts = dt + A.t_exp * (((float)ss + 0.5f) * inv_ss - 0.5f);
                float g[9];
                f += point_grad(c, dts, n_ep, A.max_iter, &bad, g);
#pragma unroll
                for (int j = 0; j < 9; ++j) gp[j] += g[j];
            }
            f *= inv_ss;
#pragma unroll
            for (int j = 0; j < 9; ++j) gp[j] *= inv_ss;
        }
        if (A.flux) A.flux[(size_t)v * A.n_t + i] = f;
        float res = f - yi;
        acc[9] = fmaf(wi * res, res, acc[9]);
        float tw = 2.0f * wi * res;
#pragma unroll
        for (int j = 0; j < 9; ++j) acc[j] = fmaf(tw, gp[j], acc[j]);
        }
    }
    if (bad) atomicAdd(&sbad, 1);
    // deterministic block reduction (the skipped tiles' sums in FP64)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ssr_out += __shfl_xor_sync(0xffffffffu, ssr_out, o);
    if (lane == 0) sout[warp] = ssr_out;
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        float x = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sred[warp][j] = x;
    }
    __syncthreads();
    __syncthreads();
    if (threadIdx.x < 10) {
        float x = 0.0f;
        for (int w = 0; w < TB / 32; ++w) x += sred[w][threadIdx.x];
        if (threadIdx.x < 9) {
            A.grad[(size_t)v * 9 + threadIdx.x] = x;
        } else if (A.ssr) {
            double so = 0.0;
            for (int w = 0; w < TB / 32; ++w) so += sout[w];
            A.ssr[v] = (float)((double)x + so);
        }
    }
    if (threadIdx.x == 0 && sbad && A.n_bad) atomicAdd(A.n_bad, sbad);
}

}  // namespace

extern "C" {

// work buffer: [n_t] time split, then per tile of TT times its time range
// and its residual sum with the flux at 1, each part 256-byte aligned
static size_t bwd_split_bytes(int n_t) { return ((size_t)n_t * sizeof(float2) + 255) & ~(size_t)255; }
static size_t bwd_tiles(int n_t) { return ((size_t)n_t + TT - 1) / TT; }

size_t pt_ma_quad_bwd_work_bytes(int n_t)
{
    if (n_t <= 0) return 256;
    const size_t nt = bwd_tiles(n_t);
    return bwd_split_bytes(n_t) + ((nt * sizeof(float2) + 255) & ~(size_t)255) + ((nt * sizeof(double) + 255) & ~(size_t)255);
}

int pt_ma_quad_bwd(const double *t, int n_t, const pt_theta *th, int n_ss, double t_exp, int max_iter,
                   const float *y, const float *wt, float *grad, float *ssr, float *flux, void *work,
                   size_t work_bytes, int *n_bad, pt_stream_t stream)
{
    if (!th || th->n_v < 0 || n_t < 0 || n_ss < 1 || n_ss > 256 || max_iter < 1 || max_iter > 64)
        return PT_ERR_ARG;
    if (!(t_exp >= 0.0 && t_exp < 1.0e30))
        return pt_internal::set_error(PT_ERR_DOMAIN, "pt_ma_quad_bwd", "exposure time must be finite and >= 0");
    if (n_t == 0 || th->n_v == 0) return PT_OK;
    if (!th->t0 || !th->P || !th->a || !th->b || !th->k || !th->u1 || !th->u2) return PT_ERR_ARG;
    if ((th->e == nullptr) != (th->w == nullptr)) return PT_ERR_ARG;
    if (!t || !y || !grad) return PT_ERR_ARG;
    if (!work) return PT_ERR_WORKSPACE;
    if (work_bytes < pt_ma_quad_bwd_work_bytes(n_t)) return PT_ERR_WORKSPACE;
    if (th->n_v > 0x7fffffff) return PT_ERR_ARG;
    if (((uintptr_t)work & 15u) != 0u)
        return pt_internal::set_error(PT_ERR_WORKSPACE, "pt_ma_quad_bwd", "work buffer must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nt = bwd_tiles(n_t);
    float2 *ts = (float2 *)work;
    float2 *tmm = (float2 *)((char *)work + bwd_split_bytes(n_t));
    double *tssr = (double *)((char *)tmm + ((nt * sizeof(float2) + 255) & ~(size_t)255));
    tile_kernel<<<(unsigned)nt, TT, 0, s>>>(t, y, wt, n_t, ts, tmm, tssr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pt_internal::set_error(PT_ERR_CUDA, "tile_kernel", cudaGetErrorString(e));
    BwdArgs A;
    A.tsplit = ts;
    A.tile_mm = tmm;
    A.tile_ssr = tssr;
    A.n_t = n_t;
    A.th = *th;
    A.n_ss = n_ss;
    A.t_exp = (float)t_exp;
    A.max_iter = max_iter;
    A.y = y;
    A.wt = wt;
    A.grad = grad;
    A.ssr = ssr;
    A.flux = flux;
    A.n_bad = n_bad;
    ma_bwd_kernel<<<th->n_v, TB, 0, s>>>(A);
    e = cudaGetLastError();
    return e == cudaSuccess ? PT_OK : pt_internal::set_error(PT_ERR_CUDA, "ma_bwd_kernel", cudaGetErrorString(e));
}

}  // extern "C"
