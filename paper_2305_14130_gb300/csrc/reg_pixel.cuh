// Consistency term of the extended model at one pixel (eqs. 8, 11, 12), shared by
// the plan's kernel and the allocation-free one.  Over the ns components:
//   B = sum b_i;  c_s = (1 - b_s)/(B - b_s) inside sink_s else 0;  d_s = b_s inside else 1
//   (W m)_s = (d_s - c_s b_s) m_s + c_s sum_i b_i m_i              (eq. 11)
//   omega_s = b'_s / sum b'                                        (eq. 12)
//   r = (I - 1 omega^T) W m;  phi += 1/2 eta^2 |r|^2
//   y = r - omega (1^T r);  g_i += eta^2 [(d_i - c_i b_i) y_i + b_i sum_s c_s y_s]
// The residual r and the norm are FP64 (r is the small difference of nearly equal
// components).  Outside every sinkhole of the pixel W is the identity, so the
// common case needs no division, no pass for sum_s c_s y_s and only a few FP64
// operations per component (GB300's FP64 rate bounds this code).
#pragma once

#include <cstdint>

namespace efwi {

// General pixel (some component has its sinkhole here), FP64 throughout.
__device__ __forceinline__ double reg_pixel_sink(const float *__restrict__ m, const float *__restrict__ b,
                                                 const float *__restrict__ bp, const uint8_t *__restrict__ sink,
                                                 int ns, long long npix, long long p, double eta2, float *g) {
    double B = 0, BM = 0, SBp = 0;
    for (int s = 0; s < ns; ++s) {
        const long long o = s * npix + p;
        const double bs = b[o];
        B += bs;
        BM += bs * (double)m[o];
        SBp += bp[o];
    }
    // (W m)_s with c_s and d_s - c_s b_s (0 and 1 outside sink_s)
    auto wm = [&](long long o, double &c, double &dc) -> double {
        const double ms = m[o];
        c = 0.0;
        dc = 1.0;
        if (sink[o] != 0) {
            const double bs = b[o];
            c = (1.0 - bs) / (B - bs);
            dc = bs - c * bs;
            return dc * ms + c * BM;
        }
        return ms;
    };
    double mean = 0.0;
    for (int s = 0; s < ns; ++s) {
        const long long o = s * npix + p;
        double c, dc;
        mean += (double)bp[o] * wm(o, c, dc);
    }
    mean /= SBp;
    double R = 0, acc = 0;
    for (int s = 0; s < ns; ++s) {
        double c, dc;
        const double r = wm(s * npix + p, c, dc) - mean;
        acc += r * r;
        R += r;
    }
    if (!g) return acc;
    const double Rw = R / SBp;                        // omega_s (1^T r) = b'_s Rw
    double CY = 0;
    for (int s = 0; s < ns; ++s) {
        const long long o = s * npix + p;
        double c, dc;
        const double r = wm(o, c, dc) - mean;
        CY += c * (r - (double)bp[o] * Rw);
    }
    for (int s = 0; s < ns; ++s) {
        const long long o = s * npix + p;
        double c, dc;
        const double y = (wm(o, c, dc) - mean) - (double)bp[o] * Rw;
        g[o] = (float)((double)g[o] + eta2 * (dc * y + (double)b[o] * CY));
    }
    return acc;
}

// Returns sum_s r_s^2 of pixel p; adds the gradient into g (skipped when g is null).
// Where no component has its sinkhole, W = I (d_s = 1, c_s = 0): r_s = m_s - mean
// with mean = sum b'_s m_s / sum b', formed in FP64 (the norm's residual); the
// gradient y_s = r_s - b'_s (1^T r) / sum b' is added to the FP32 g in FP32.
__device__ __forceinline__ double reg_pixel(const float *__restrict__ m, const float *__restrict__ b,
                                            const float *__restrict__ bp, const uint8_t *__restrict__ sink, int ns,
                                            long long npix, long long p, double eta2, float *g) {
    double SBp = 0, SBpM = 0;
    bool any = false;
    for (int s = 0; s < ns; ++s) {
        const long long o = s * npix + p;
        const double bps = bp[o];
        SBp += bps;
        SBpM = fma(bps, (double)m[o], SBpM);
        any |= sink[o] != 0;
    }
    if (any && ns > 1) return reg_pixel_sink(m, b, bp, sink, ns, npix, p, eta2, g);
    const double mean = SBpM / SBp;
    double R = 0, acc = 0;
    for (int s = 0; s < ns; ++s) {
        const double r = (double)m[s * npix + p] - mean;
        acc = fma(r, r, acc);
        R += r;
    }
    if (g) {
        const float Rw = (float)(R / SBp), e2 = (float)eta2;
        for (int s = 0; s < ns; ++s) {
            const long long o = s * npix + p;
            const float y = (float)((double)m[o] - mean) - bp[o] * Rw;
            g[o] = g[o] + e2 * y;
        }
    }
    return acc;
}

}  // namespace efwi
