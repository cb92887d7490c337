// Exact line minimum of the quartic E(x) = c0 + c1 x + c2 x^2 + c3 x^3 + c4 x^4
// (the exact line search of the Introduction), shared by every CG form.
//
// Rule: among the real roots of E'(x) with positive curvature, the lowest E
// wins; ties go to the smaller |x|, then to x > 0.  With c4 < 0 (the Kim
// functional with eta inside the gap, where H' has positive eigenvalues) the
// quartic is unbounded below and only its local minima are candidates.  No
// candidate, or c4 = c3 = 0 with c2 <= 0, is OMM_ERR_LINESEARCH; non-finite
// data is OMM_ERR_NONFINITE.
//
// The roots of E' = 4c4 x^3 + 3c3 x^2 + 2c2 x + c1 are found by one warp:
// multisection on the Cauchy bracket (-R, R) -- every round the 32 lanes
// evaluate the cubic at 32 interior points and keep the first sign change, so
// the bracket shrinks 33-fold without a division -- then deflation, a stable
// quadratic formula for the other two roots and Newton polishing, one root per
// lane.  A dependent FP64 operation takes ~64 cycles on this part (FP32: ~4),
// so the bracketing and the deflation run in FP32 on the cubic scaled to
// t = x / R with coefficients of magnitude <= 1, and only the polishing runs in
// FP64: Newton steps whose reciprocal of E'' is taken in FP32 (each step then
// shrinks the error by ~1e-7, so two or three reach FP64 precision from the
// FP32 root).  Where the scaling leaves the FP32 range the FP64 multisection
// runs instead.
#pragma once

#include <math.h>

#include "omm_internal.cuh"

namespace omm {
namespace lm {

__device__ __forceinline__ double quartic_val(const double *c, double x) {
    return c[0] + x * (c[1] + x * (c[2] + x * (c[3] + x * c[4])));
}

// Choose the minimiser among the candidate roots r[0 .. nr).
__device__ __forceinline__ int select_min(const double *c, const double *r, int nr, double *xout) {
    bool have = false;
    double best = 0.0, bestv = 0.0;
    for (int pass = 0; pass < 2 && !have; ++pass)
        for (int i = 0; i < nr; ++i) {
            const double x = r[i];
            if (!isfinite(x)) continue;
            const double curv = 12.0 * c[4] * x * x + 6.0 * c[3] * x + 2.0 * c[2];
            if (pass == 0 && !(curv > 0.0)) continue;
            if (pass == 1 && !(c[4] > 0.0)) continue;
            const double v = quartic_val(c, x);
            if (!have || v < bestv || (v == bestv && (fabs(x) < fabs(best) || (fabs(x) == fabs(best) && x > best)))) {
                have = true;
                best = x;
                bestv = v;
            }
        }
    if (!have) return OMM_ERR_LINESEARCH;
    *xout = best;
    return OMM_OK;
}

// Cases that need no cubic root: fills r/nr or returns a status; returns -1
// when the cubic (c4 > 0) must be solved.
__device__ __forceinline__ int trivial_cases(const double *c, double *r, int *nr, double *xout, bool *done) {
    *done = true;
    for (int i = 0; i < 5; ++i)
        if (!isfinite(c[i])) return OMM_ERR_NONFINITE;
    if (c[4] == 0.0 && c[3] == 0.0) {
        if (c[2] > 0.0) {
            *xout = -c[1] / (2.0 * c[2]);
            return OMM_OK;
        }
        return OMM_ERR_LINESEARCH;
    }
    *done = false;
    *nr = 0;
    if (c[4] == 0.0) {   // c3 != 0: E' = 3 c3 x^2 + 2 c2 x + c1
        const double a = 3.0 * c[3], b = 2.0 * c[2], cc = c[1];
        const double disc = b * b - 4.0 * a * cc;
        if (disc >= 0.0) {
            const double sq = sqrt(disc);
            const double t = -0.5 * (b + (b >= 0.0 ? sq : -sq));
            if (t != 0.0) {
                r[(*nr)++] = t / a;
                r[(*nr)++] = cc / t;
            }
        }
        *done = true;
        return select_min(c, r, *nr, xout);
    }
    return -1;
}

// Deflate a x^3 + b x^2 + c x + d by the root x1 and add the quadratic's roots.
__device__ __forceinline__ int deflate(double a, double b, double c, double x1, double *r) {
    int nr = 0;
    r[nr++] = x1;
    const double p = b + a * x1, q = c + p * x1;   // (x - x1)(a x^2 + p x + q)
    const double disc = p * p - 4.0 * a * q;
    if (disc >= 0.0) {
        const double sq = sqrt(disc);
        const double t = -0.5 * (p + (p >= 0.0 ? sq : -sq));
        if (t != 0.0) {
            r[nr++] = t / a;
            r[nr++] = q / t;
        } else {
            r[nr++] = 0.0;
        }
    }
    return nr;
}

__device__ __forceinline__ double polish(double a, double b, double c, double d, double x) {
    auto f = [&](double t) { return ((a * t + b) * t + c) * t + d; };
    auto fp = [&](double t) { return (3.0 * a * t + 2.0 * b) * t + c; };
    for (int it = 0; it < 3; ++it) {
        const double dx = fp(x);
        if (dx == 0.0) break;
        const double xn = x - f(x) / dx;
        if (!isfinite(xn)) break;
        if (fabs(f(xn)) <= fabs(f(x))) x = xn; else break;
    }
    return x;
}

// FP64 Newton polish of a root of a x^3 + b x^2 + c x + d; the step's
// reciprocal derivative is taken in FP32 where it is representable.
__device__ __forceinline__ double polish_fast(double a, double b, double c, double d, double x) {
    auto f = [&](double t) { return ((a * t + b) * t + c) * t + d; };
    auto fp = [&](double t) { return (3.0 * a * t + 2.0 * b) * t + c; };
    double fx = f(x);
    for (int it = 0; it < 6; ++it) {
        if (fx == 0.0) break;
        const double dx = fp(x);
        if (dx == 0.0) break;
        const float rf = 1.0f / (float)dx;
        const double step = (isfinite(rf) && rf != 0.0f) ? fx * (double)rf : fx / dx;
        const double xn = x - step;
        if (!isfinite(xn)) break;
        const double fn = f(xn);
        if (!(fabs(fn) < fabs(fx))) break;
        x = xn;
        fx = fn;
        if (fabs(step) <= 1e-17 * fabs(x)) break;
    }
    return x;
}

// FP64 multisection (the form used where the scaled cubic leaves the FP32 range).
__device__ inline int quartic_min_warp64(const double *c, double *xout) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    double r[3];
    int nr = 0;
    bool done;
    const int st = trivial_cases(c, r, &nr, xout, &done);
    if (done) return st;
    // E' with a positive leading coefficient (negated when c4 < 0: same roots)
    const double sg = c[4] > 0.0 ? 1.0 : -1.0;
    const double a = sg * 4.0 * c[4], b = sg * 3.0 * c[3], cc = sg * 2.0 * c[2], d = sg * c[1];
    auto f = [&](double t) { return ((a * t + b) * t + cc) * t + d; };
    const double R = 1.0 + fmax(fabs(b), fmax(fabs(cc), fabs(d))) / a;
    double lo = -R, hi = R;   // f(lo) < 0 < f(hi): a > 0 and every root lies inside
    const double step = 1.0 / 33.0;
    for (int round = 0; round < 64; ++round) {
        const double w = hi - lo;
        if (!(w > 4e-16 * fmax(1.0, fmax(fabs(lo), fabs(hi))))) break;
        const double xl = lo + w * ((double)(lane + 1) * step);
        const double fl = f(xl);
        const unsigned nonneg = __ballot_sync(full, !(fl < 0.0));   // first lane with f >= 0 closes the bracket
        const int j = nonneg ? __ffs(nonneg) - 1 : 32;
        const double xprev = __shfl_sync(full, xl, j > 0 ? j - 1 : 0);
        const double xj = __shfl_sync(full, xl, j < 32 ? j : 31);
        const double nlo = j > 0 ? xprev : lo, nhi = j < 32 ? xj : hi;
        if (nlo == lo && nhi == hi) break;
        lo = nlo;
        hi = nhi;
    }
    nr = deflate(a, b, cc, 0.5 * (lo + hi), r);
    // one root per lane for the polishing, then everyone takes all of them
    double mine = lane < nr ? polish(a, b, cc, d, r[lane]) : 0.0;
    for (int i = 0; i < nr; ++i) r[i] = __shfl_sync(full, mine, i);
    return select_min(c, r, nr, xout);
}

// Warp form: all 32 lanes of one warp call it with the same c; every lane
// gets the same status and x.
__device__ inline int quartic_min_warp(const double *c, double *xout) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    double r[3];
    int nr = 0;
    bool done;
    const int st = trivial_cases(c, r, &nr, xout, &done);
    if (done) return st;
    const double sg = c[4] > 0.0 ? 1.0 : -1.0;
    const double a = sg * 4.0 * c[4], b = sg * 3.0 * c[3], cc = sg * 2.0 * c[2], d = sg * c[1];
    // Cauchy bound R = 1 + max(|b|, |cc|, |d|) / a, kept an upper bound of the FP32 quotient
    const float qf = (float)fmax(fabs(b), fmax(fabs(cc), fabs(d))) / (float)a;
    if (!(qf >= 0.0f) || !isfinite(qf) || qf > 1e30f) return quartic_min_warp64(c, xout);
    const double R = 1.0 + (double)qf * (1.0 + 1e-5);
    // the cubic in t = x / R, scaled so that its largest coefficient is 1
    const double A = a * R * R * R, B = b * R * R, C = cc * R, D = d;
    const float inv = 1.0f / (float)fmax(fmax(fabs(A), fabs(B)), fmax(fabs(C), fabs(D)));
    if (!isfinite(inv) || inv == 0.0f) return quartic_min_warp64(c, xout);
    const float Af = (float)A * inv, Bf = (float)B * inv, Cf = (float)C * inv, Df = (float)D * inv;
    auto g = [&](float t) { return fmaf(fmaf(fmaf(Af, t, Bf), t, Cf), t, Df); };
    float lo = -1.0f, hi = 1.0f;   // g(-1) < 0 < g(1): every root lies inside
    const float step = 1.0f / 33.0f;
    for (int round = 0; round < 24; ++round) {
        const float w = hi - lo;
        if (!(w > 2e-7f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f)) break;
        const float tl = fmaf(w, (float)(lane + 1) * step, lo);
        const float gl = g(tl);
        const unsigned nonneg = __ballot_sync(full, !(gl < 0.0f));   // first lane with g >= 0 closes the bracket
        const int j = nonneg ? __ffs(nonneg) - 1 : 32;
        const float tprev = __shfl_sync(full, tl, j > 0 ? j - 1 : 0);
        const float tj = __shfl_sync(full, tl, j < 32 ? j : 31);
        const float nlo = j > 0 ? tprev : lo, nhi = j < 32 ? tj : hi;
        if (nlo == lo && nhi == hi) break;
        lo = nlo;
        hi = nhi;
    }
    // deflate in FP32: (t - t1)(Af t^2 + p t + q)
    const float t1 = 0.5f * (lo + hi);
    float tr[3] = {t1, 0.0f, 0.0f};
    nr = 1;
    const float p = fmaf(Af, t1, Bf), q = fmaf(p, t1, Cf);
    const float disc = fmaf(p, p, -4.0f * Af * q);
    if (disc >= 0.0f) {
        const float sq = sqrtf(disc);
        const float t = -0.5f * (p + (p >= 0.0f ? sq : -sq));
        if (t != 0.0f) {
            tr[nr++] = t / Af;
            tr[nr++] = q / t;
        } else {
            tr[nr++] = 0.0f;
        }
    } else if (disc > -1e-5f * p * p) {
        tr[nr++] = -0.5f * p / Af;   // a double root within the FP32 rounding
    }
    // one root per lane for the FP64 polishing, then everyone takes all of them
    const float tmine = lane == 0 ? tr[0] : lane == 1 ? tr[1] : tr[2];
    const double mine = lane < nr ? polish_fast(a, b, cc, d, (double)tmine * R) : 0.0;
    for (int i = 0; i < nr; ++i) r[i] = __shfl_sync(full, mine, i);
    return select_min(c, r, nr, xout);
}

}  // namespace lm
}  // namespace omm
