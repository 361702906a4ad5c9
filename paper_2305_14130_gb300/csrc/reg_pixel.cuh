// Consistency term of the extended model at one pixel (eqs. 8, 11, 12), shared by
// the plan's kernel and the allocation-free one.  Over the ns components:
//   B = sum b_i;  c_s = (1 - b_s)/(B - b_s) inside sink_s else 0;  d_s = b_s inside else 1
//   (W m)_s = (d_s - c_s b_s) m_s + c_s sum_i b_i m_i              (eq. 11)
//   omega_s = b'_s / sum b'                                        (eq. 12)
//   r = (I - 1 omega^T) W m;  phi += 1/2 eta^2 |r|^2
//   y = r - omega (1^T r);  g_i += eta^2 [(d_i - c_i b_i) y_i + b_i sum_s c_s y_s]
// FP64 arithmetic: r is the small difference of nearly equal components.  Outside
// every sinkhole of the pixel W is the identity, so the common case needs no
// division and no pass for sum_s c_s y_s (GB300's FP64 rate bounds this code).
#pragma once

#include <cstdint>

namespace efwi {

// Returns sum_s r_s^2 of pixel p; adds the gradient into g (skipped when g is null).
__device__ __forceinline__ double reg_pixel(const float *__restrict__ m, const float *__restrict__ b,
                                            const float *__restrict__ bp, const uint8_t *__restrict__ sink, int ns,
                                            long long npix, long long p, double eta2, float *g) {
    double B = 0, BM = 0, SBp = 0, SBpM = 0;
    bool any = false;
    for (int s = 0; s < ns; ++s) {
        const long long o = s * npix + p;
        const double bs = b[o], ms = m[o], bps = bp[o];
        B += bs;
        BM += bs * ms;
        SBp += bps;
        SBpM += bps * ms;
        any |= sink[o] != 0;
    }
    any = any && ns > 1;
    // (W m)_s with c_s and d_s - c_s b_s (0 and 1 outside sink_s)
    auto wm = [&](long long o, double &c, double &dc) -> double {
        const double ms = m[o];
        c = 0.0;
        dc = 1.0;
        if (any && sink[o] != 0) {
            const double bs = b[o];
            c = (1.0 - bs) / (B - bs);
            dc = bs - c * bs;
            return dc * ms + c * BM;
        }
        return ms;
    };
    double mean = SBpM;                               // sum_s b'_s (W m)_s, W = I
    if (any) {
        mean = 0.0;
        for (int s = 0; s < ns; ++s) {
            const long long o = s * npix + p;
            double c, dc;
            mean += (double)bp[o] * wm(o, c, dc);
        }
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
    if (any)
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
        const double cy = any ? (double)b[o] * CY : 0.0;
        g[o] = (float)((double)g[o] + eta2 * (dc * y + cy));
    }
    return acc;
}

}  // namespace efwi
