// Pseudo-Hessian of the paper's illumination-compensation comparison method
// (pseudo-Hessian = diagonal of the approximate Hessian; the paper builds it by
// auto-correlating the absolute particle velocity wavefields in time, summing
// over shots, clipping and scaling, and hands it to l-BFGS as the initial
// inverse-Hessian guess):
//   H(x) = sum_s sum_n |v_s(x, t_{n+1/2})|^2,
// with |v|^2 at a node from the mean of the two staggered neighbours of each
// component (vx at i -+ 1/2, vz at j -+ 1/2), and the clipped, scaled inverse
//   P(x) = c / max(H(x), c),  c = eps * max_x H   (P = 1 everywhere if H = 0).
//
// k_vel_energy runs after every forward step and adds |v|^2 of every physical
// node of every shot, in FP32, to a Kahan-compensated FP32 sum with the
// wavefield layout (the same precision as the imaging sums); k_ph_collect adds
// the compensated sums of the shots covering each physical pixel in FP64
// (fixed shot order) and takes block maxima; k_max_final and k_ph_scale finish
// the inverse.
#include <algorithm>

#include "plan.hpp"

namespace efwi {
namespace {

constexpr int kT = 256;

// grid (ceil(wmax / kT), nz, ns): one thread per physical node of shot blockIdx.z
__global__ void k_vel_energy(const ShotDev *shots, Fields F, float *sum, float *cmp) {
    const ShotDev &s = shots[blockIdx.z];
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= s.w) return;
    const long long c = cell_of(s, i + s.P, (int)blockIdx.y + s.P);
    const float vx = 0.5f * (F.vx[c - 1] + F.vx[c]);
    const float vz = 0.5f * (F.vz[c - s.pitch] + F.vz[c]);
    // Kahan (1965) compensated add; cmp holds the part of sum that overshoots
    const float y = (vx * vx + vz * vz) - cmp[c];
    const float t = sum[c] + y;
    cmp[c] = (t - sum[c]) - y;
    sum[c] = t;
}

__device__ double block_max(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

__global__ void k_ph_collect(const ShotDev *shots, int ns, const float *sum, const float *cmp, int nx,
                             long long npix, float *h, double *partial) {
    double m = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < npix;
         k += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(k / nx), i = (int)(k - (long long)j * nx);
        double v = 0.0;
        for (int s = 0; s < ns; ++s) {
            const ShotDev &sh = shots[s];
            const int il = i - sh.x0;
            if (il >= 0 && il < sh.w) {
                const long long c = cell_of(sh, il + sh.P, j + sh.P);
                v += (double)sum[c] - (double)cmp[c];
            }
        }
        h[k] = (float)v;
        m = fmax(m, v);
    }
    m = block_max(m);
    if (threadIdx.x == 0) partial[blockIdx.x] = m;
}

__global__ void k_max_final(const double *partial, int n, double *out) {
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v = fmax(v, partial[k]);
    v = block_max(v);
    if (threadIdx.x == 0) *out = v;
}

__global__ void k_ph_scale(const float *h, long long npix, const double *hmax, double eps, float *hinv) {
    const double c = eps * *hmax;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < npix;
         k += (long long)gridDim.x * blockDim.x)
        hinv[k] = c > 0.0 ? (float)(c / fmax((double)h[k], c)) : 1.f;
}

}  // namespace

void launch_vel_energy(efwi_plan *p, Fields F, float *sum, float *cmp, cudaStream_t st) {
    int wmax = 1;
    for (int s = 0; s < p->d.ns; ++s) wmax = std::max(wmax, p->shots[s].w);
    const dim3 grid((wmax + kT - 1) / kT, p->d.nz, p->d.ns);
    k_vel_energy<<<grid, kT, 0, st>>>(p->shots_d, F, sum, cmp);
    p->launches++;
}

void launch_ph_finish(efwi_plan *p, const float *sum, const float *cmp, double eps, float *h, float *hinv,
                      cudaStream_t st) {
    const long long npix = (long long)p->d.nx * p->d.nz;
    k_ph_collect<<<kPartials, kT, 0, st>>>(p->shots_d, p->d.ns, sum, cmp, p->d.nx, npix, h, p->partial);
    k_max_final<<<1, 1024, 0, st>>>(p->partial, kPartials, p->partial + kPartials);
    p->launches += 2;
    if (hinv) {
        k_ph_scale<<<kPartials, kT, 0, st>>>(h, npix, p->partial + kPartials, eps, hinv);
        p->launches++;
    }
}

}  // namespace efwi
