// Kernels around the stencils: material preparation, moment-tensor injection,
// DAS sampling and its transpose, FP64 misfit, chain rule to (Vp, Vs, rho),
// Kahan folding of per-segment imaging sums, wavefield checkpoints (FP32 or
// scaled FP16/BF16), zone-of-influence weights and the consistency term.
#include <algorithm>
#include <cmath>

#include "plan.hpp"
#include "reg_pixel.cuh"

namespace efwi {
namespace {

constexpr int kRedThreads = 256;

// --------------------------------------------------------------------------
// Materials (model m of eq. 1; one extended component per shot).
// --------------------------------------------------------------------------
struct MatArgs {
    const ShotDev *shots;
    const float *vp, *vs, *rho, *ref;   // model [ns][nz][nx]; ref [3][nz][nx]
    Mat M;                              // outputs (const-cast inside)
    int nx, nz, shot;
    int *err;                           // device flag: bit 2 set for a non-finite or invalid model value
    int shear;                          // a gradient call: flag mu <= 0 where the chain rule divides by it
                                        // (1: stress-form adjoint) or where the scaled-stress adjoint's
                                        // sums are converted, also lambda + mu <= 0 (2) (EFWI_FLAG_SHEAR)
};

__device__ void model_at(const MatArgs &a, const ShotDev &s, int shot, int i, int j, float &vp, float &vs,
                         float &rho) {
    i = min(i, s.NX - 1);
    j = min(j, s.NZ - 1);
    int ix = i - s.P, iz = j - s.P;
    const bool phys = ix >= 0 && ix < s.w && iz >= 0 && iz < a.nz;
    ix = min(max(ix, 0), s.w - 1) + s.x0;
    iz = min(max(iz, 0), a.nz - 1);
    const long long k = (long long)iz * a.nx + ix;
    if (phys) {
        const long long o = (long long)shot * a.nz * a.nx + k;
        vp = a.vp[o]; vs = a.vs[o]; rho = a.rho[o];
    } else {
        const long long n = (long long)a.nz * a.nx;
        vp = a.ref[k]; vs = a.ref[n + k]; rho = a.ref[2 * n + k];
    }
}

// FP32 arithmetic (each operation rounded once: the library builds without
// multiply-add contraction); the inputs are FP32 already.
__global__ void k_materials(MatArgs a) {
    const int shot = a.shot >= 0 ? a.shot : blockIdx.z;
    const ShotDev s = a.shots[shot];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= s.NX || j >= s.NZ) return;
    float vp, vs, rho, mu[4], r[4];
    const int di[4] = {0, 1, 0, 1}, dj[4] = {0, 0, 1, 1};
    for (int k = 0; k < 4; ++k) {
        model_at(a, s, shot, i + di[k], j + dj[k], vp, vs, rho);
        mu[k] = rho * vs * vs;
        r[k] = rho;
    }
    model_at(a, s, shot, i, j, vp, vs, rho);
    // a non-finite velocity or density, or a non-positive density, makes the call's results invalid
    if (!(isfinite(vp) && isfinite(vs) && isfinite(rho) && rho > 0.f)) atomicOr(a.err, EFWI_FLAG_BAD_MODEL);
    const long long c = cell_of(s, i, j);
    const bool zero = mu[0] == 0.f || mu[1] == 0.f || mu[2] == 0.f || mu[3] == 0.f;
    const float lam = rho * (vp * vp - 2.f * vs * vs);
    // the chain rule divides by mu on the physical nodes (the harmonic mean's derivative);
    // the scaled-stress adjoint's sums are divided by 2 (lambda + mu), 2 mu and mu_xz on the
    // physical nodes and the half cells next to them (nodes P-1 .. P+w, P-1 .. NZ-P)
    if (a.shear) {
        const int lo = a.shear == 2 ? s.P - 1 : s.P;
        if (i >= lo && i <= s.P + s.w - (a.shear == 2 ? 0 : 1) && j >= lo &&
            j <= s.NZ - s.P - (a.shear == 2 ? 0 : 1) && !(mu[0] > 0.f && (a.shear == 1 || lam + mu[0] > 0.f)))
            atomicOr(a.err, EFWI_FLAG_SHEAR);
    }
    ((float *)a.M.lam)[c] = lam;
    ((float *)a.M.mu)[c] = mu[0];
    ((float *)a.M.muxz)[c] = zero ? 0.f : 4.f / (1.f / mu[0] + 1.f / mu[1] + 1.f / mu[2] + 1.f / mu[3]);
    ((float *)a.M.bx)[c] = 0.5f * (1.f / r[0] + 1.f / r[1]);
    ((float *)a.M.bz)[c] = 0.5f * (1.f / r[0] + 1.f / r[2]);
}

// --------------------------------------------------------------------------
// Moment-tensor source (eq. 2): sigma^{n+1} -= M (w_{n+1} - w_n) delta_h.
// --------------------------------------------------------------------------
__global__ void k_inject(const ShotDev *shots, Fields F, const float *dw, int nt, int n, int s0, int ns) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns) return;
    const int s = s0 + t;
    const ShotDev sh = shots[s];
    const float w = dw[(long long)s * nt + n];
    for (int q = 0; q < 4; ++q) {
        F.sxx[sh.off + sh.inj_n[q]] -= sh.mxx * w * sh.inj_nw[q];
        F.szz[sh.off + sh.inj_n[q]] -= sh.mzz * w * sh.inj_nw[q];
        F.sxz[sh.off + sh.inj_x[q]] -= sh.mxz * w * sh.inj_xw[q];
    }
}

// Vector-force source (eq. 2, second case), after the velocity sub-step of
// step n: v^{n+1/2} += dt b F w_n delta_h on the vx and vz grids.  The fused
// steps add the same term, with the same expression, inside their velocity phase.
__global__ void k_force(const ShotDev *shots, Fields F, Mat M, const float *wv, int nt, int n, int s0, int ns,
                        float dt, float *segx, float *segz) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns) return;
    const int s = s0 + t;
    const ShotDev sh = shots[s];
    const float w = wv[(long long)s * nt + n];
    for (int q = 0; q < 4; ++q) {
        const long long cx = sh.off + sh.inj_vx[q], cz = sh.off + sh.inj_vz[q];
        F.vx[cx] = F.vx[cx] + dt * M.bx[cx] * (sh.fx * w * sh.inj_vxw[q]);
        F.vz[cz] = F.vz[cz] + dt * M.bz[cz] * (sh.fz * w * sh.inj_vzw[q]);
    }
    if (segx)                                   // the segment copy of v^{n+1/2} (after all four corners)
        for (int q = 0; q < 4; ++q) {
            segx[sh.off + sh.inj_vx[q]] = F.vx[sh.off + sh.inj_vx[q]];
            segz[sh.off + sh.inj_vz[q]] = F.vz[sh.off + sh.inj_vz[q]];
        }
}

// --------------------------------------------------------------------------
// DAS sampling K_r (eq. 3): strain rate of trace t = sum of 16 weighted
// velocity samples (weights carry +-t_k / L); strain = running time integral.
// --------------------------------------------------------------------------
__global__ void k_das_fwd(const ShotDev *shots, const int *tr_shot, const int *tr_off, const float *tr_w,
                          double *acc, const float *vx, const float *vz, float *d, int t0, int ntr, int nt, int n,
                          float dt, int strain) {
    const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= t0 + ntr) return;
    const long long base = shots[tr_shot[t]].off;
    float rate = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float *f = (k >> 2) & 1 ? vz : vx;
        rate += tr_w[t * 16 + k] * f[base + tr_off[t * 16 + k]];
    }
    float out = rate;
    if (strain) {
        const double a = acc[t] + (double)dt * rate;
        acc[t] = a;
        out = (float)a;
    }
    d[(long long)t * nt + n] = out;
}

// Adjoint source of step n: coefficient of trace t (reverse cumulative residual for strain).
__global__ void k_das_adj_prep(const float *resid, double *acc, float *coef, int t0, int ntr, int nt, int n, float dt,
                               int strain) {
    const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= t0 + ntr) return;
    const float r = resid[(long long)t * nt + n];
    if (strain) {
        const double a = acc[t] + r;
        acc[t] = a;
        coef[t] = (float)((double)dt * a);
    } else {
        coef[t] = r;
    }
}

// Transposed sampling as a deterministic gather over the cells touched by gauge
// ends; also the b-imaging contribution of this adjoint increment.
__global__ void k_das_adj_gather(const ShotDev *shots, GatherCSR g, const float *coef, Fields A, const float *vfx,
                                 const float *vfz, SnapR sr, float *Gbx, float *Gbz, int g0, int gn) {
    const int k = g0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g0 + gn) return;
    float inc = 0.f;
    for (int e = g.ptr[k]; e < g.ptr[k + 1]; ++e) inc += g.w[e] * coef[g.tr[e]];
    const int shot = g.tgt_shot[k];
    const long long c = shots[shot].off + g.tgt_off[k];
    if (g.tgt_field[k] == 0) {
        A.vx[c] += inc;
        const float v = sr.h ? snap_get_rt(sr.h, c, sr.kind) * snap_scale_down(sr.hmax, 0, shot, sr.ns) : vfx[c];
        Gbx[c] += v * inc;
    } else {
        A.vz[c] += inc;
        const float v = sr.h ? snap_get_rt(sr.h, sr.F + c, sr.kind) * snap_scale_down(sr.hmax, 1, shot, sr.ns) : vfz[c];
        Gbz[c] += v * inc;
    }
}

// --------------------------------------------------------------------------
// Residual and FP64 misfit (eq. 4): deterministic two-level reduction.
// --------------------------------------------------------------------------
__device__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

__global__ void k_residual(const float *d, const float *dobs, float *r, long long n, double *partial) {
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double x = (double)d[k] - (double)dobs[k];
        r[k] = (float)x;
        acc += x * x;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void k_final_sum(const double *partial, int n, double scale, double *out, int accumulate) {
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += partial[k];
    v = block_sum(v);
    if (threadIdx.x == 0) *out = (accumulate ? *out : 0.0) + scale * v;
}

// --------------------------------------------------------------------------
// Chain rule: imaging sums for (lambda, mu, mu_xz, b_x, b_z) -> (Vp, Vs, rho).
//   lambda = rho (Vp^2 - 2 Vs^2), mu = rho Vs^2,
//   d mu_xz / d mu_k = mu_xz^2 / (4 mu_k^2) over its 4 nodes,
//   d b / d rho_k = -1 / (2 rho_k^2) over its 2 nodes; G_b holds b * dphi/db.
// --------------------------------------------------------------------------
struct ChainArgs {
    const ShotDev *shots;
    const float *vp, *vs, *rho, *mask;
    Mat M;
    const float *Glam, *Gmu, *Gmuxz, *Gbx, *Gbz;
    float *gvp, *gvs, *grho;
    int nx, nz;
};

// FP32 arithmetic; mu_xz / mu is formed before squaring so no intermediate
// leaves the range of the moduli.
__global__ void k_chain(ChainArgs a) {
    const int shot = blockIdx.z;
    const ShotDev s = a.shots[shot];
    const int ixw = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ixw >= s.w || iz >= a.nz) return;
    const int ix = ixw + s.x0;
    const long long o = ((long long)shot * a.nz + iz) * a.nx + ix;
    const float vp = a.vp[o], vs = a.vs[o], rho = a.rho[o];
    const float mu = rho * vs * vs;
    const long long c = cell_of(s, ixw + s.P, iz + s.P);
    const long long P = s.pitch;
    const float dlam = a.Glam[c];
    float dmu = a.Gmu[c];
    const long long cx[4] = {c, c - 1, c - P, c - P - 1};
    for (int k = 0; k < 4; ++k) {
        const float q = a.M.muxz[cx[k]] / mu;
        dmu += a.Gmuxz[cx[k]] * (0.25f * q * q);
    }
    const float db = a.Gbx[c] / a.M.bx[c] + a.Gbx[c - 1] / a.M.bx[c - 1] + a.Gbz[c] / a.M.bz[c] +
                     a.Gbz[c - P] / a.M.bz[c - P];
    const float drho = -((0.5f * db) / rho) / rho;
    float gvp = 2.f * rho * vp * dlam;
    float gvs = 2.f * rho * vs * (dmu - 2.f * dlam);
    float grh = dlam * (vp * vp - 2.f * vs * vs) + dmu * (vs * vs) + drho;
    if (a.mask) {
        const float m = a.mask[(long long)iz * a.nx + ix];
        gvp *= m; gvs *= m; grh *= m;
    }
    a.gvp[o] = gvp;
    a.gvs[o] = gvs;
    a.grho[o] = grh;
}

// Kahan (1965) compensated add of the segment sums into the totals.
__global__ void k_kahan(float *G, float *tot, float *cmp, long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float y = G[k] - cmp[k];
        const float t = tot[k] + y;
        cmp[k] = (t - tot[k]) - y;
        tot[k] = t;
        G[k] = 0.f;
    }
}

// --------------------------------------------------------------------------
// Checkpoints in scaled FP16 / BF16: per snapshot, per field and shot, s = max |x|
// and x stored as RNE(x 2^k) with the power of two of store_exp(s).
// --------------------------------------------------------------------------
// grid-stride pieces shared by the checkpoint kernels and the store self-test
__device__ __forceinline__ void absmax_span(const float *x, long long n, float *s) {
    float m = 0.f;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[k]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((int *)s, __float_as_int(m));   // non-negative floats order as ints
}

template <class T>
__device__ __forceinline__ void pack_span(const float *x, long long n, float s, T *y) {
    const float up = pow2f(store_exp(s));
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        y[k] = to_store<T>(x[k] * up);
}

template <class T>
__device__ __forceinline__ void unpack_span(const T *y, long long n, float s, float *x) {
    const float down = pow2f(-store_exp(s));
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        x[k] = from_store(y[k]) * down;
}

__global__ void k_absmax(const ShotDev *shots, const float *fields, long long F, float *scale, int ns) {
    const int f = blockIdx.y, shot = blockIdx.z;
    const ShotDev s = shots[shot];
    const long long n = (long long)(s.NZ + 2 * EFWI_GZ) * s.pitch;
    absmax_span(fields + f * F + s.off, n, &scale[f * ns + shot]);
}

template <class T>
__global__ void k_pack(const ShotDev *shots, const float *fields, long long F, const float *scale, T *out, int ns) {
    const int f = blockIdx.y, shot = blockIdx.z;
    const ShotDev s = shots[shot];
    const long long n = (long long)(s.NZ + 2 * EFWI_GZ) * s.pitch;
    pack_span<T>(fields + f * F + s.off, n, scale[f * ns + shot], out + f * F + s.off);
}

template <class T>
__global__ void k_unpack(const ShotDev *shots, float *fields, long long F, const float *scale, const T *in, int ns) {
    const int f = blockIdx.y, shot = blockIdx.z;
    const ShotDev s = shots[shot];
    const long long n = (long long)(s.NZ + 2 * EFWI_GZ) * s.pitch;
    unpack_span<T>(in + f * F + s.off, n, scale[f * ns + shot], fields + f * F + s.off);
}

// The reduced-precision snapshot of the velocities of state buffer `vx, vz` (the
// last step of a pass, which no later step stages): per shot (blockIdx.z) and
// field (blockIdx.y) the whole block with the maxima its step accumulated.
template <class T>
__global__ void k_snap_tail(const ShotDev *shots, const float *vx, const float *vz, SnapW sw) {
    const int f = blockIdx.y, shot = blockIdx.z;
    const ShotDev s = shots[shot];
    const long long n = (long long)(s.NZ + 2 * EFWI_GZ) * s.pitch;
    const float mx = sw.hmax[(long long)(f * sw.ns + shot) * kMaxPad];
    pack_span<T>((f ? vz : vx) + s.off, n, mx, static_cast<T *>(sw.h) + f * sw.F + s.off);
}

// Self-test kernels: one array as one snapshot field.
__global__ void k_selftest_absmax(const float *x, long long n, float *s) { absmax_span(x, n, s); }
template <class T>
__global__ void k_selftest_pack(const float *x, long long n, const float *s, T *y) { pack_span<T>(x, n, *s, y); }
template <class T>
__global__ void k_selftest_unpack(const T *y, long long n, const float *s, float *x) { unpack_span<T>(y, n, *s, x); }

// --------------------------------------------------------------------------
// Zone of influence (eq. 10) and the consistency term (eqs. 8, 11, 12).
// --------------------------------------------------------------------------
struct ZoiShot {
    double xa, xb, taper, sx, sz, ax, az;
};

__device__ double zoi_b(double r, double n, double lnnu) {
    r = fmin(fmax(r, 0.0), 1.0);
    return (pow(cos(0.5 * M_PI * r), n) - lnnu) / (1.0 - lnnu);
}

__global__ void k_zoi(ZoiShot z, int s, int nx, int nz, double dx, double dz, double n, double lnnu, float *b,
                      float *bp, uint8_t *sink) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= nx || iz >= nz) return;
    const double x = ix * dx, zz = iz * dz;
    const double dist = fmax(fmax(z.xa - x, x - z.xb), 0.0);
    const double r_out = fmin(dist / z.taper, 1.0);
    const double ex = (x - z.sx) / z.ax, ez = (zz - z.sz) / z.az;
    const double dm = sqrt(ex * ex + ez * ez);
    const bool inside = dm < 1.0;
    const double bb = fmin(zoi_b(r_out, n, lnnu), zoi_b(1.0 - dm, n, lnnu));
    const long long o = ((long long)s * nz + iz) * nx + ix;
    b[o] = (float)bb;
    bp[o] = inside ? 1.f : (float)bb;
    sink[o] = inside ? 1 : 0;
}

// Consistency term per pixel: reg_pixel (reg_pixel.cuh).
// Collapse of an extended field to one physical field (eq. 9, and eq. 15 when
// applied to the per-source gradients): out = S_w W x~ per pixel, FP64:
//   (W x)_s = (d_s - c_s b_s) x_s + c_s sum_i b_i x_i  (eq. 11, c_s and d_s as in k_reg)
//   out = sum_s b'_s (W x)_s / sum_s b'_s               (eq. 12)
__global__ void k_collapse(const float *x, const float *b, const float *bp, const uint8_t *sink, int ns,
                           long long npix, float *out) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
        double B = 0, BX = 0, SBp = 0;
        for (int s = 0; s < ns; ++s) {
            const long long o = s * npix + p;
            B += b[o]; BX += (double)b[o] * x[o]; SBp += bp[o];
        }
        double acc = 0;
        for (int s = 0; s < ns; ++s) {
            const long long o = s * npix + p;
            const double bs = b[o];
            const bool in = sink[o] != 0 && ns > 1;
            const double c = in ? (1.0 - bs) / (B - bs) : 0.0;
            const double dd = in ? bs : 1.0;
            acc += (double)bp[o] * ((dd - c * bs) * x[o] + c * BX);
        }
        out[p] = (float)(acc / SBp);
    }
}

__global__ void k_reg(const float *m, const float *b, const float *bp, const uint8_t *sink, int ns, long long npix,
                      double eta2, float *g, double *partial) {
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x)
        acc += reg_pixel(m, b, bp, sink, ns, npix, p, eta2, g);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

}  // namespace

// ==========================================================================
// Launchers
// ==========================================================================

void launch_materials(efwi_plan *p, const float *vp, const float *vs, const float *rho, cudaStream_t st,
                      int gradient) {
    MatArgs a{p->shots_d, vp, vs, rho, p->ref, materials(p), p->d.nx, p->d.nz, -1, p->dev_err,
              !gradient ? 0 : p->adj_form == EFWI_ADJ_FORM_SCALED ? 2 : 1};
    dim3 b(32, 8);
    dim3 g((p->max_nx + 31) / 32, (p->nzp + 7) / 8, p->d.ns);
    k_materials<<<g, b, 0, st>>>(a);
    p->launches++;
}

void launch_inject(efwi_plan *p, Fields F, int n, int shot, cudaStream_t st) {
    const int s0 = shot < 0 ? 0 : shot, cnt = shot < 0 ? p->d.ns : 1;
    k_inject<<<(cnt + 127) / 128, 128, 0, st>>>(p->shots_d, F, p->dw, p->d.nt, n, s0, cnt);
    p->launches++;
}

void launch_force(efwi_plan *p, Fields F, int n, int shot, float *segx, float *segz, cudaStream_t st) {
    if (!p->has_force) return;
    const int s0 = shot < 0 ? 0 : shot, cnt = shot < 0 ? p->d.ns : 1;
    k_force<<<(cnt + 127) / 128, 128, 0, st>>>(p->shots_d, F, materials(p), p->wv, p->d.nt, n, s0, cnt,
                                               (float)p->d.dt, segx, segz);
    p->launches++;
}

void launch_das_fwd(efwi_plan *p, Fields F, int n, float *d, int shot, cudaStream_t st) {
    const int t0 = shot < 0 ? 0 : p->shots[shot].tr0;
    const int cnt = shot < 0 ? p->d.ntr : p->shots[shot].ntr;
    if (cnt == 0) return;
    k_das_fwd<<<(cnt + 127) / 128, 128, 0, st>>>(p->shots_d, p->tr_shot, p->tr_off, p->tr_w, p->tr_acc, F.vx, F.vz, d,
                                                 t0, cnt, p->d.nt, n, (float)p->d.dt, p->d.das_mode == EFWI_DAS_STRAIN);
    p->launches++;
}

void launch_das_adj(efwi_plan *p, Fields A, const SnapIn &si, float *Gbx, float *Gbz, int n, int shot,
                    cudaStream_t st) {
    const int t0 = shot < 0 ? 0 : p->shots[shot].tr0;
    const int cnt = shot < 0 ? p->d.ntr : p->shots[shot].ntr;
    if (cnt == 0) return;
    k_das_adj_prep<<<(cnt + 127) / 128, 128, 0, st>>>(p->resid, p->tr_acc, p->tr_coef, t0, cnt, p->d.nt, n,
                                                      (float)p->d.dt, p->d.das_mode == EFWI_DAS_STRAIN);
    const int g0 = shot < 0 ? 0 : p->gather_ptr[shot];
    const int gn = shot < 0 ? p->gather.n_tgt : p->gather_ptr[shot + 1] - p->gather_ptr[shot];
    p->launches++;
    if (gn == 0) return;
    k_das_adj_gather<<<(gn + 127) / 128, 128, 0, st>>>(p->shots_d, p->gather, p->tr_coef, A, si.fx, si.fz, si.sr,
                                                       Gbx, Gbz, g0, gn);
    p->launches++;
}

void launch_residual(efwi_plan *p, const float *d, const float *dobs, double *phi, cudaStream_t st) {
    const long long n = (long long)p->d.ntr * p->d.nt;
    k_residual<<<kPartials, kRedThreads, 0, st>>>(d, dobs, p->resid, n, p->partial);
    k_final_sum<<<1, 1024, 0, st>>>(p->partial, kPartials, 0.5, phi, 0);
    p->launches += 2;
}

void launch_chain_rule(efwi_plan *p, const float *vp, const float *vs, const float *rho, const float *const *G,
                       const float *mask, float *gvp, float *gvs, float *grho, cudaStream_t st) {
    const size_t bytes = sizeof(float) * (size_t)p->d.ns * p->d.nz * p->d.nx;
    cudaMemsetAsync(gvp, 0, bytes, st);
    cudaMemsetAsync(gvs, 0, bytes, st);
    cudaMemsetAsync(grho, 0, bytes, st);
    ChainArgs a{p->shots_d, vp, vs, rho, mask, materials(p), G[0], G[1], G[2], G[3], G[4], gvp, gvs, grho,
                p->d.nx, p->d.nz};
    dim3 b(32, 8);
    int wmax = 0;
    for (auto &s : p->shots) wmax = wmax > s.w ? wmax : s.w;
    dim3 g((wmax + 31) / 32, (p->d.nz + 7) / 8, p->d.ns);
    k_chain<<<g, b, 0, st>>>(a);
    p->launches++;
}

void launch_kahan_fold(efwi_plan *p, cudaStream_t st) {
    k_kahan<<<4 * 152, 256, 0, st>>>(p->G, p->Gtot, p->Gcmp, 5 * p->fsz_total);
    p->launches++;
}

void launch_ckpt_save(efwi_plan *p, int slot, cudaStream_t st) {
    const long long F = p->fsz_total, H = p->H;
    const int ns = p->d.ns;
    float *dst = p->ck.psi + (size_t)slot * 2 * H;
    cudaMemcpyAsync(dst, psi_block(p->psi, p, p->psi_v), sizeof(float) * H, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(dst + H, psi_block(p->psi, p, 2 + p->psi_s), sizeof(float) * H, cudaMemcpyDeviceToDevice, st);
    const float *src = p->state[p->scur];
    if (p->ck.store == EFWI_STORE_FP32) {
        cudaMemcpyAsync((float *)p->ck.fields + (size_t)slot * 5 * F, src, sizeof(float) * 5 * F,
                        cudaMemcpyDeviceToDevice, st);
        return;
    }
    float *sc = p->ck.scale + (size_t)slot * 5 * ns;
    cudaMemsetAsync(sc, 0, sizeof(float) * 5 * ns, st);
    dim3 g(64, 5, ns);
    k_absmax<<<g, 256, 0, st>>>(p->shots_d, src, F, sc, ns);
    if (p->ck.store == EFWI_STORE_FP16)
        k_pack<__half><<<g, 256, 0, st>>>(p->shots_d, src, F, sc, (__half *)p->ck.fields + (size_t)slot * 5 * F, ns);
    else
        k_pack<__nv_bfloat16><<<g, 256, 0, st>>>(p->shots_d, src, F, sc,
                                                  (__nv_bfloat16 *)p->ck.fields + (size_t)slot * 5 * F, ns);
    p->launches += 2;
}

void launch_snap_tail(efwi_plan *p, const SnapW &sw, cudaStream_t st) {
    const Fields F = state_fields(p, p->scur);
    dim3 g(64, 2, p->d.ns);
    if (sw.kind == EFWI_STORE_FP16) k_snap_tail<__half><<<g, 256, 0, st>>>(p->shots_d, F.vx, F.vz, sw);
    else k_snap_tail<__nv_bfloat16><<<g, 256, 0, st>>>(p->shots_d, F.vx, F.vz, sw);
    p->launches++;
}

void launch_ckpt_load(efwi_plan *p, int slot, cudaStream_t st) {
    const long long F = p->fsz_total, H = p->H;
    const int ns = p->d.ns;
    const float *srcp = p->ck.psi + (size_t)slot * 2 * H;
    cudaMemcpyAsync(psi_block(p->psi, p, p->psi_v), srcp, sizeof(float) * H, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(psi_block(p->psi, p, 2 + p->psi_s), srcp + H, sizeof(float) * H, cudaMemcpyDeviceToDevice, st);
    float *dst = p->state[p->scur];
    if (p->ck.store == EFWI_STORE_FP32) {
        cudaMemcpyAsync(dst, (const float *)p->ck.fields + (size_t)slot * 5 * F, sizeof(float) * 5 * F,
                        cudaMemcpyDeviceToDevice, st);
        return;
    }
    const float *sc = p->ck.scale + (size_t)slot * 5 * ns;
    dim3 g(64, 5, ns);
    if (p->ck.store == EFWI_STORE_FP16)
        k_unpack<__half><<<g, 256, 0, st>>>(p->shots_d, dst, F, sc,
                                            (const __half *)p->ck.fields + (size_t)slot * 5 * F, ns);
    else
        k_unpack<__nv_bfloat16><<<g, 256, 0, st>>>(p->shots_d, dst, F, sc,
                                                    (const __nv_bfloat16 *)p->ck.fields + (size_t)slot * 5 * F, ns);
    p->launches++;
}

int launch_zoi(int ns, int nx, int nz, double dx, double dz, const efwi_zoi_desc *z, float *b, float *bp,
               uint8_t *sink, cudaStream_t st, std::string &err) {
    if (ns < 1 || nx < 1 || nz < 1 || !(dx > 0) || !(dz > 0) || !z || !b || !bp || !sink) {
        err = "bad arguments to efwi_zoi_weights";
        return EFWI_ERR_ARG;
    }
    if (!z->active_x || !z->taper || !z->sink_xz || !z->sink_axes || !(z->nu > 0 && z->nu < 1) || !(z->n > 0)) {
        err = "bad zone-of-influence description (need 0 < nu < 1, n > 0)";
        return EFWI_ERR_ARG;
    }
    for (int s = 0; s < ns; ++s) {
        ZoiShot zs{z->active_x[2 * s], z->active_x[2 * s + 1], z->taper[s], z->sink_xz[2 * s], z->sink_xz[2 * s + 1],
                   z->sink_axes[2 * s], z->sink_axes[2 * s + 1]};
        if (!(zs.taper > 0) || !(zs.ax > 0) || !(zs.az > 0)) {
            err = "taper and sinkhole axes must be > 0";
            return EFWI_ERR_ARG;
        }
        dim3 bl(32, 8), g((nx + 31) / 32, (nz + 7) / 8);
        k_zoi<<<g, bl, 0, st>>>(zs, s, nx, nz, dx, dz, z->n, std::log(z->nu), b, bp, sink);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return EFWI_ERR_CUDA;
    }
    return EFWI_OK;
}

void launch_collapse(int ns, long long npix, const float *x, const float *b, const float *bp, const uint8_t *sink,
                     float *out, cudaStream_t st) {
    const long long blocks = std::min<long long>((npix + 255) / 256, 152LL * 16);
    k_collapse<<<(int)std::max<long long>(blocks, 1), 256, 0, st>>>(x, b, bp, sink, ns, npix, out);
}

void launch_reg(efwi_plan *p, const float *m, const float *b, const float *bp, const uint8_t *sink, double eta,
                double *phi, float *g, int accumulate_phi, cudaStream_t st, int ns) {
    const long long npix = (long long)p->d.nz * p->d.nx;
    k_reg<<<kPartials, kRedThreads, 0, st>>>(m, b, bp, sink, ns > 0 ? ns : p->d.ns, npix, eta * eta, g, p->partial);
    k_final_sum<<<1, 1024, 0, st>>>(p->partial, kPartials, 0.5 * eta * eta, phi, accumulate_phi);
    p->launches += 2;
}

}  // namespace efwi

// --------------------------------------------------------------------------
// Numerics self-tests: the reduced-precision store and the Kahan fold on
// caller arrays, through the device routines the time loops use.
// --------------------------------------------------------------------------
extern "C" int efwi_selftest_store(int store, long long n, const float *x, void *enc, float *y, float *s_out,
                                   efwi_stream_t stream) {
    using namespace efwi;
    if (n < 1 || !x || !y || !s_out || (store != EFWI_STORE_FP32 && !enc) || store < EFWI_STORE_FP32 ||
        store > EFWI_STORE_BF16) {
        set_thread_error("efwi_selftest_store: n >= 1, x, y, s_out (and enc for FP16/BF16) required");
        return EFWI_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(s_out, 0, sizeof(float), st);
    const int g = (int)std::min<long long>((n + 255) / 256, 4 * 152);
    k_selftest_absmax<<<g, 256, 0, st>>>(x, n, s_out);
    if (store == EFWI_STORE_FP32) {
        cudaMemcpyAsync(y, x, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
    } else if (store == EFWI_STORE_FP16) {
        k_selftest_pack<__half><<<g, 256, 0, st>>>(x, n, s_out, (__half *)enc);
        k_selftest_unpack<__half><<<g, 256, 0, st>>>((const __half *)enc, n, s_out, y);
    } else {
        k_selftest_pack<__nv_bfloat16><<<g, 256, 0, st>>>(x, n, s_out, (__nv_bfloat16 *)enc);
        k_selftest_unpack<__nv_bfloat16><<<g, 256, 0, st>>>((const __nv_bfloat16 *)enc, n, s_out, y);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(std::string("efwi_selftest_store: ") + cudaGetErrorString(e));
        return EFWI_ERR_CUDA;
    }
    return EFWI_OK;
}

extern "C" int efwi_selftest_kahan(long long n, int nterms, float *terms, float *tot, float *cmp,
                                   efwi_stream_t stream) {
    using namespace efwi;
    if (n < 1 || nterms < 1 || !terms || !tot || !cmp) {
        set_thread_error("efwi_selftest_kahan: n, nterms >= 1 and non-NULL arrays required");
        return EFWI_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(tot, 0, sizeof(float) * n, st);
    cudaMemsetAsync(cmp, 0, sizeof(float) * n, st);
    const int g = (int)std::min<long long>((n + 255) / 256, 4 * 152);
    for (int k = 0; k < nterms; ++k) k_kahan<<<g, 256, 0, st>>>(terms + (size_t)k * n, tot, cmp, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(std::string("efwi_selftest_kahan: ") + cudaGetErrorString(e));
        return EFWI_ERR_CUDA;
    }
    return EFWI_OK;
}
