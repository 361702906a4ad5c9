// Limited-memory BFGS on the device, with a strong-Wolfe line search and the
// convergence rate of eq. 13 as stopping rule (the optimizer of the paper's
// inversions: l-BFGS with a step length satisfying the Wolfe conditions).
//
// Vectors (the model x, gradients, the m stored pairs s_i = x_{i+1} - x_i,
// y_i = g_{i+1} - g_i) are FP32 device arrays of n elements; every inner
// product is an FP64 reduction with a fixed summation order (deterministic).
// The search direction is the two-loop recursion (Nocedal & Wright, Alg. 7.4)
// with H_0 = gamma I, gamma = s^T y / y^T y of the newest pair, or, when the
// caller sets a positive diagonal D as the initial guess (the paper hands its
// l-BFGS an approximate inverse pseudo-Hessian), H_0 = gamma D with
// gamma = s^T y / y^T D y (H_0 = D without pairs); its scalars
// (alpha_i, beta) stay on the device, so the recursion is a fixed sequence of
// launches.  The line search (Nocedal & Wright, Alg. 3.5 with the zoom of
// Alg. 3.6, quadratic interpolation safeguarded to the inner 80 % of the
// bracket, else bisection) is scalar control on the host: it reads phi and
// g^T d of every trial point, which the caller's objective returns.
#include <cmath>
#include <string>
#include <vector>

#include "plan.hpp"

namespace {

constexpr int kLbThreads = 256;
constexpr int kLbBlocks = 1024;                 // FP64 partials of one inner product

__device__ double lb_block_sum(double v) {
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

// partial[b] = sum over block b's grid-stride share of x_i y_i
__global__ void k_dot(const float *x, const float *y, long long n, double *partial) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)x[i] * (double)y[i];
    acc = lb_block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// out = scale * sum(partial) [* (*mul) when mul]; the single final block keeps the order fixed
__global__ void k_dot_final(const double *partial, int nb, double scale, const double *mul, double *out) {
    double v = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) v += partial[k];
    v = lb_block_sum(v);
    if (threadIdx.x == 0) *out = scale * v * (mul ? *mul : 1.0);
}

// partial[b] = sum over block b's grid-stride share of x_i w_i y_i
__global__ void k_dot3(const float *x, const float *w, const float *y, long long n, double *partial) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)x[i] * ((double)w[i] * (double)y[i]);
    acc = lb_block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// y = w * y elementwise
__global__ void k_mul(float *y, const float *w, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = w[i] * y[i];
}

// y += (a0 - a1) * x, with a0, a1 device scalars (a1 may be NULL)
__global__ void k_axpy_dev(float *y, const float *x, long long n, const double *a0, const double *a1, double sign) {
    const double a = sign * (*a0 - (a1 ? *a1 : 0.0));
    const float af = (float)a;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = y[i] + af * x[i];
}

// y = a * x (a device scalar times sign)
__global__ void k_scale_dev(float *y, const float *x, long long n, const double *a, double sign) {
    const float af = (float)(sign * *a);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = af * x[i];
}

// out = x + alpha * d (alpha a host scalar)
__global__ void k_trial(float *out, const float *x, const float *d, long long n, float alpha) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = x[i] + alpha * d[i];
}

// out = a - b
__global__ void k_sub(float *out, const float *a, const float *b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

// rho = 1 / sy and gamma = sy / yy from the scalars of the new pair
__global__ void k_pair_scalars(const double *sy, const double *yy, double *rho, double *gamma) {
    *rho = 1.0 / *sy;
    *gamma = *sy / *yy;
}

}  // namespace

struct efwi_lbfgs {
    long long n = 0;
    int m = 0;
    std::vector<int> order;           // slots of the stored pairs, oldest first (at most m)
    float *S = nullptr, *Y = nullptr; // (m + 1) x n: the stored pairs and one candidate slot
    float *d = nullptr, *xt = nullptr, *gt = nullptr;
    float *D = nullptr;               // diagonal initial inverse Hessian (efwi_lbfgs_set_h0)
    bool has_d = false;
    double *dev = nullptr;            // device scalars, see the offsets below
    double *partial = nullptr;
    double c1 = 1e-4, c2 = 0.9;
    int max_ls = 20;
    double step0 = 0;                 // first trial length without pairs (0: min(1, 1 / ||d||))
    // device-resident line search (efwi_lbfgs_iterate_device): its state, the trial point's
    // phi and phi', a capture stream and the graph of the last (objective, x, phi, g)
    void *ls_state = nullptr;
    double *ls_phit = nullptr;
    cudaStream_t ls_cap = nullptr;
    cudaGraphExec_t ls_exec = nullptr;
    const void *ls_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int slots() const { return m + 1; }
    // device scalar offsets: rho[m + 1], alpha[m + 1], then the ones below
    int o_rho() const { return 0; }
    int o_alpha() const { return slots(); }
    int o_beta() const { return 2 * slots(); }
    int o_gamma() const { return 2 * slots() + 1; }
    int o_tmp() const { return 2 * slots() + 2; }
    int o_sy() const { return 2 * slots() + 3; }
    int o_yy() const { return 2 * slots() + 4; }
    int nscal() const { return 2 * slots() + 5; }
    // a slot holding no stored pair
    int free_slot() const {
        for (int k = 0; k < slots(); ++k) {
            bool used = false;
            for (int o : order) used = used || o == k;
            if (!used) return k;
        }
        return 0;
    }
};

namespace {

__global__ void k_neg(float *y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = -y[i];
}

int lb_grid(long long n) {
    const long long b = (n + kLbThreads - 1) / kLbThreads;
    return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 8));
}

// *out = scale * x^T y [* *mul]; a fixed grid of kLbBlocks blocks keeps the order fixed for every n
void dot_dev(efwi_lbfgs *h, const float *x, const float *y, double *out, double scale, const double *mul,
             cudaStream_t st) {
    k_dot<<<kLbBlocks, kLbThreads, 0, st>>>(x, y, h->n, h->partial);
    k_dot_final<<<1, 1024, 0, st>>>(h->partial, kLbBlocks, scale, mul, out);
}

int read_scalar(const double *p, double *v, cudaStream_t st) {
    if (cudaMemcpyAsync(v, p, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return EFWI_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return EFWI_ERR_CUDA;
    return EFWI_OK;
}

float *slot_s(efwi_lbfgs *h, int k) { return h->S + (long long)k * h->n; }
float *slot_y(efwi_lbfgs *h, int k) { return h->Y + (long long)k * h->n; }

// d = -H g by the two-loop recursion; H = H_0 (I or D) without stored pairs
void lb_direction(efwi_lbfgs *h, const float *g, cudaStream_t st) {
    const long long n = h->n;
    const int G = lb_grid(n);
    double *rho = h->dev + h->o_rho(), *alpha = h->dev + h->o_alpha(), *beta = h->dev + h->o_beta();
    cudaMemcpyAsync(h->d, g, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
    const int np = (int)h->order.size();
    for (int j = np - 1; j >= 0; --j) {                          // newest to oldest
        const int k = h->order[j];
        dot_dev(h, slot_s(h, k), h->d, alpha + k, 1.0, rho + k, st);
        k_axpy_dev<<<G, kLbThreads, 0, st>>>(h->d, slot_y(h, k), n, alpha + k, nullptr, -1.0);
    }
    if (np > 0) k_scale_dev<<<G, kLbThreads, 0, st>>>(h->d, h->d, n, h->dev + h->o_gamma(), 1.0);
    if (h->has_d) k_mul<<<G, kLbThreads, 0, st>>>(h->d, h->D, n);
    for (int j = 0; j < np; ++j) {                               // oldest to newest
        const int k = h->order[j];
        dot_dev(h, slot_y(h, k), h->d, beta, 1.0, rho + k, st);
        k_axpy_dev<<<G, kLbThreads, 0, st>>>(h->d, slot_s(h, k), n, alpha + k, beta, 1.0);
    }
    k_neg<<<G, kLbThreads, 0, st>>>(h->d, n);
}

struct Trial {
    double a = 0, phi = 0, dphi = 0;
};

struct Search {
    efwi_lbfgs *h;
    const float *x;
    efwi_objective_fn fn;
    void *ctx;
    cudaStream_t st;
    double phi0 = 0, dphi0 = 0;
    int evals = 0, rc = EFWI_OK;

    // phi and phi' at x + a d (the trial point and its gradient stay in xt, gt)
    bool eval(double a, Trial &t) {
        if (evals >= h->max_ls) return false;
        ++evals;
        k_trial<<<lb_grid(h->n), kLbThreads, 0, st>>>(h->xt, x, h->d, h->n, (float)a);
        double phi = 0;
        const int r = fn(ctx, h->xt, &phi, h->gt, (efwi_stream_t)st);
        if (r != 0) {
            rc = r < 0 ? r : EFWI_ERR_ARG;
            efwi::set_thread_error("l-BFGS: the objective callback returned " + std::to_string(r));
            return false;
        }
        double *tmp = h->dev + h->o_tmp();
        dot_dev(h, h->gt, h->d, tmp, 1.0, nullptr, st);
        if (read_scalar(tmp, &t.dphi, st) != EFWI_OK) {
            rc = EFWI_ERR_CUDA;
            efwi::set_thread_error("l-BFGS: reading g^T d failed");
            return false;
        }
        t.a = a;
        t.phi = phi;
        // a trial whose objective or slope is not finite (a step long enough to make
        // the modelling unstable) fails sufficient decrease: phi = +inf, so that it
        // bounds the bracket from above and the zoom bisects towards the shorter step
        if (!std::isfinite(phi) || !std::isfinite(t.dphi)) t.phi = HUGE_VAL;
        return true;
    }
    bool armijo_fails(const Trial &t) const { return t.phi > phi0 + h->c1 * t.a * dphi0; }
    bool curvature_holds(const Trial &t) const { return std::fabs(t.dphi) <= -h->c2 * dphi0; }

    // quadratic through phi(lo), phi'(lo), phi(hi), kept inside the inner 80 % of the bracket
    static double interp(const Trial &lo, const Trial &hi) {
        const double w = hi.a - lo.a;
        const double den = 2.0 * (hi.phi - lo.phi - lo.dphi * w);
        double a = den > 0 ? lo.a - lo.dphi * w * w / den : lo.a + 0.5 * w;
        const double lower = std::fmin(lo.a, hi.a) + 0.1 * std::fabs(w);
        const double upper = std::fmax(lo.a, hi.a) - 0.1 * std::fabs(w);
        if (!(a >= lower && a <= upper)) a = lo.a + 0.5 * w;
        return a;
    }

    // Alg. 3.6: the bracket [lo, hi] holds a step satisfying the strong Wolfe conditions
    bool zoom(Trial lo, Trial hi, Trial &out) {
        for (;;) {
            Trial t;
            if (!eval(interp(lo, hi), t)) return false;
            if (armijo_fails(t) || t.phi >= lo.phi) {
                hi = t;
            } else {
                if (curvature_holds(t)) {
                    out = t;
                    return true;
                }
                if (t.dphi * (hi.a - lo.a) >= 0) hi = lo;
                lo = t;
            }
        }
    }

    // Alg. 3.5: increase the step until a bracket is found or the conditions hold
    bool run(double a0, Trial &out) {
        Trial prev;
        prev.a = 0;
        prev.phi = phi0;
        prev.dphi = dphi0;
        double a = a0;
        for (int i = 1;; ++i) {
            Trial t;
            if (!eval(a, t)) return false;
            if (armijo_fails(t) || (i > 1 && t.phi >= prev.phi)) return zoom(prev, t, out);
            if (curvature_holds(t)) {
                out = t;
                return true;
            }
            if (t.dphi >= 0) return zoom(t, prev, out);
            a = extrapolate(prev, t);
            prev = t;
        }
    }

    // next bracketing trial after t (sufficient decrease holds, phi'(t) < 0): the zero
    // of the secant of phi' through prev and t when phi' increased (the minimiser of a
    // quadratic), kept within [2 a, 10 a]; 2 a otherwise
    static double extrapolate(const Trial &prev, const Trial &t) {
        const double a = t.a;
        if (t.dphi > prev.dphi) {
            const double sec = a - t.dphi * (a - prev.a) / (t.dphi - prev.dphi);
            return std::fmin(std::fmax(sec, 2.0 * a), 10.0 * a);
        }
        return 2.0 * a;
    }
};

// ---------------------------------------------------------------------------
// The line search of Search::run / Search::zoom as a device state machine: the
// same steps, tests and interpolation in the same FP64 arithmetic, one trial
// point per call of k_ls_step, so that a CUDA graph can repeat
// (trial point, objective, phi', step) in a conditional while-node with no host
// synchronisation until the search ends.
// ---------------------------------------------------------------------------
struct LsTrial {
    double a, phi, dphi;
};

struct LsState {
    double phi0, dphi0, c1, c2;
    double a;                    // the step of the next trial point
    LsTrial prev, lo, hi, out;
    int phase;                   // 0: bracketing (Alg. 3.5), 1: zoom (Alg. 3.6)
    int i;                       // bracketing iteration, from 1
    int evals, max_ls;
    int done, ok;                // search over; a step satisfying the strong Wolfe conditions found
};

__device__ double ls_interp(const LsTrial &lo, const LsTrial &hi) {
    const double w = hi.a - lo.a;
    const double den = 2.0 * (hi.phi - lo.phi - lo.dphi * w);
    double a = den > 0 ? lo.a - lo.dphi * w * w / den : lo.a + 0.5 * w;
    const double lower = fmin(lo.a, hi.a) + 0.1 * fabs(w);
    const double upper = fmax(lo.a, hi.a) - 0.1 * fabs(w);
    if (!(a >= lower && a <= upper)) a = lo.a + 0.5 * w;
    return a;
}

// Search::extrapolate
__device__ double ls_extrapolate(const LsTrial &prev, const LsTrial &t) {
    const double a = t.a;
    if (t.dphi > prev.dphi) {
        const double sec = a - t.dphi * (a - prev.a) / (t.dphi - prev.dphi);
        return fmin(fmax(sec, 2.0 * a), 10.0 * a);
    }
    return 2.0 * a;
}

__global__ void k_ls_init(LsState *s, double phi0, double dphi0, double a0, double c1, double c2, int max_ls) {
    LsState t{};
    t.phi0 = phi0;
    t.dphi0 = dphi0;
    t.c1 = c1;
    t.c2 = c2;
    t.a = a0;
    t.prev = LsTrial{0.0, t.phi0, t.dphi0};
    t.phase = 0;
    t.i = 1;
    t.max_ls = max_ls;
    *s = t;
}

// out = x + a d with the step a of the search state
__global__ void k_trial_state(float *out, const float *x, const float *d, long long n, const LsState *s) {
    const float alpha = (float)s->a;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = x[i] + alpha * d[i];
}

__global__ void k_ls_step(LsState *st, const double *phit, const double *dphit, cudaGraphConditionalHandle cond) {
    LsState s = *st;
    if (!s.done) {
        s.evals += 1;
        LsTrial t{s.a, *phit, *dphit};
        if (!isfinite(t.phi) || !isfinite(t.dphi)) t.phi = HUGE_VAL;   // as in Search::eval
        const bool armijo_fails = t.phi > s.phi0 + s.c1 * t.a * s.dphi0;
        const bool curvature = fabs(t.dphi) <= -s.c2 * s.dphi0;
        if (s.phase == 0) {
            if (armijo_fails || (s.i > 1 && t.phi >= s.prev.phi)) {
                s.lo = s.prev; s.hi = t; s.phase = 1;
            } else if (curvature) {
                s.out = t; s.done = 1; s.ok = 1;
            } else if (t.dphi >= 0) {
                s.lo = t; s.hi = s.prev; s.phase = 1;
            } else {
                s.a = ls_extrapolate(s.prev, t); s.prev = t; s.i += 1;
            }
            if (!s.done && s.phase == 1) s.a = ls_interp(s.lo, s.hi);
        } else {
            if (armijo_fails || t.phi >= s.lo.phi) {
                s.hi = t;
            } else if (curvature) {
                s.out = t; s.done = 1; s.ok = 1;
            } else {
                if (t.dphi * (s.hi.a - s.lo.a) >= 0) s.hi = s.lo;
                s.lo = t;
            }
            if (!s.done) s.a = ls_interp(s.lo, s.hi);
        }
        if (!s.done && s.evals >= s.max_ls) s.done = 1;   // no step within max_ls evaluations
    }
    *st = s;
    cudaGraphSetConditional(cond, s.done ? 0u : 1u);
}

}  // namespace

using efwi::set_thread_error;

namespace {

int lb_fail(int code, const std::string &msg) {
    set_thread_error(msg);
    return code;
}

int lb_check(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lb_fail(EFWI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return EFWI_OK;
}

// stores the pair (s, y) already written in the free slot k when s^T y > 0
int lb_accept_pair(efwi_lbfgs *h, int k, cudaStream_t st, int *accepted) {
    double *sy = h->dev + h->o_sy(), *yy = h->dev + h->o_yy();
    dot_dev(h, slot_s(h, k), slot_y(h, k), sy, 1.0, nullptr, st);
    if (h->has_d) {                                  // y^T D y for gamma of H_0 = gamma D
        k_dot3<<<kLbBlocks, kLbThreads, 0, st>>>(slot_y(h, k), h->D, slot_y(h, k), h->n, h->partial);
        k_dot_final<<<1, 1024, 0, st>>>(h->partial, kLbBlocks, 1.0, nullptr, yy);
    } else {
        dot_dev(h, slot_y(h, k), slot_y(h, k), yy, 1.0, nullptr, st);
    }
    double v = 0, w = 0;
    if (read_scalar(sy, &v, st) != EFWI_OK || read_scalar(yy, &w, st) != EFWI_OK)
        return lb_fail(EFWI_ERR_CUDA, "l-BFGS: reading s^T y failed");
    *accepted = 0;
    if (!(v > 0.0) || !(w > 0.0) || !std::isfinite(v) || !std::isfinite(w)) return EFWI_OK;   // curvature fails: skip
    k_pair_scalars<<<1, 1, 0, st>>>(sy, yy, h->dev + h->o_rho() + k, h->dev + h->o_gamma());
    h->order.push_back(k);
    if ((int)h->order.size() > h->m) h->order.erase(h->order.begin());
    *accepted = 1;
    return lb_check("l-BFGS pair");
}

}  // namespace

extern "C" int efwi_lbfgs_create(efwi_lbfgs **out, long long n, int m, double c1, double c2, int max_ls) {
    if (!out) return lb_fail(EFWI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || m < 1 || m > 64) return lb_fail(EFWI_ERR_ARG, "need n >= 1 and 1 <= m <= 64");
    if (!(c1 > 0 && c1 < c2 && c2 < 1)) return lb_fail(EFWI_ERR_ARG, "need 0 < c1 < c2 < 1");
    if (max_ls < 1) return lb_fail(EFWI_ERR_ARG, "max_ls must be >= 1");
    efwi_lbfgs *h = new efwi_lbfgs();
    h->n = n;
    h->m = m;
    h->c1 = c1;
    h->c2 = c2;
    h->max_ls = max_ls;
    bool ok = cudaMalloc((void **)&h->S, sizeof(float) * n * h->slots()) == cudaSuccess &&
              cudaMalloc((void **)&h->Y, sizeof(float) * n * h->slots()) == cudaSuccess &&
              cudaMalloc((void **)&h->d, sizeof(float) * n) == cudaSuccess &&
              cudaMalloc((void **)&h->xt, sizeof(float) * n) == cudaSuccess &&
              cudaMalloc((void **)&h->gt, sizeof(float) * n) == cudaSuccess &&
              cudaMalloc((void **)&h->dev, sizeof(double) * h->nscal()) == cudaSuccess &&
              cudaMalloc((void **)&h->partial, sizeof(double) * kLbBlocks) == cudaSuccess;
    if (ok) ok = cudaMemset(h->dev, 0, sizeof(double) * h->nscal()) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        efwi_lbfgs_destroy(h);
        return lb_fail(EFWI_ERR_OOM, "l-BFGS: device allocation failed");
    }
    *out = h;
    return EFWI_OK;
}

static void lb_drop_graph(efwi_lbfgs *h) {
    if (h->ls_exec) cudaGraphExecDestroy(h->ls_exec);
    h->ls_exec = nullptr;
    for (auto &k : h->ls_key) k = nullptr;
}

extern "C" int efwi_lbfgs_destroy(efwi_lbfgs *h) {
    if (!h) return EFWI_OK;
    cudaDeviceSynchronize();
    lb_drop_graph(h);
    if (h->ls_cap) cudaStreamDestroy(h->ls_cap);
    for (void *p : {(void *)h->S, (void *)h->Y, (void *)h->d, (void *)h->xt, (void *)h->gt, (void *)h->dev,
                    (void *)h->partial, (void *)h->D, h->ls_state, (void *)h->ls_phit})
        if (p) cudaFree(p);
    delete h;
    return EFWI_OK;
}

extern "C" int efwi_lbfgs_set_step0(efwi_lbfgs *h, double len) {
    if (!h || !(len >= 0) || !std::isfinite(len)) return lb_fail(EFWI_ERR_ARG, "handle NULL or len < 0");
    h->step0 = len;
    return EFWI_OK;
}

extern "C" int efwi_lbfgs_reset(efwi_lbfgs *h) {
    if (!h) return lb_fail(EFWI_ERR_ARG, "handle is NULL");
    h->order.clear();
    if (h->ls_exec) {                           // the device search's graph is captured again on next use
        cudaDeviceSynchronize();
        lb_drop_graph(h);
    }
    return EFWI_OK;
}

extern "C" int efwi_lbfgs_set_h0(efwi_lbfgs *h, const float *diag, efwi_stream_t stream) {
    if (!h) return lb_fail(EFWI_ERR_ARG, "handle is NULL");
    h->order.clear();                           // gamma of the stored pairs depends on H_0
    if (!diag) {
        h->has_d = false;
        return EFWI_OK;
    }
    if (!h->D && cudaMalloc((void **)&h->D, sizeof(float) * h->n) != cudaSuccess) {
        cudaGetLastError();
        h->D = nullptr;
        return lb_fail(EFWI_ERR_OOM, "l-BFGS: device allocation of the diagonal failed");
    }
    cudaMemcpyAsync(h->D, diag, sizeof(float) * h->n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    h->has_d = true;
    return lb_check("l-BFGS initial inverse Hessian");
}

extern "C" int efwi_lbfgs_export(efwi_lbfgs *h, int *pairs, float *S_out, float *Y_out, efwi_stream_t stream) {
    if (!h || !pairs) return lb_fail(EFWI_ERR_ARG, "NULL argument");
    *pairs = (int)h->order.size();
    if (!S_out && !Y_out) return EFWI_OK;                  // query the number of pairs only
    if (!S_out || !Y_out) return lb_fail(EFWI_ERR_ARG, "S_out and Y_out must both be given");
    cudaStream_t st = (cudaStream_t)stream;
    for (int j = 0; j < *pairs; ++j) {                      // oldest first
        const int k = h->order[j];
        cudaMemcpyAsync(S_out + (long long)j * h->n, slot_s(h, k), sizeof(float) * h->n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(Y_out + (long long)j * h->n, slot_y(h, k), sizeof(float) * h->n, cudaMemcpyDeviceToDevice, st);
    }
    return lb_check("l-BFGS export");
}

extern "C" int efwi_lbfgs_push(efwi_lbfgs *h, const float *s, const float *y, int *accepted, efwi_stream_t stream) {
    if (!h || !s || !y) return lb_fail(EFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int k = h->free_slot();
    cudaMemcpyAsync(slot_s(h, k), s, sizeof(float) * h->n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(slot_y(h, k), y, sizeof(float) * h->n, cudaMemcpyDeviceToDevice, st);
    int acc = 0;
    const int rc = lb_accept_pair(h, k, st, &acc);
    if (accepted) *accepted = acc;
    return rc;
}

extern "C" int efwi_lbfgs_direction(efwi_lbfgs *h, const float *g, float *d, efwi_stream_t stream) {
    if (!h || !g || !d) return lb_fail(EFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    lb_direction(h, g, st);
    cudaMemcpyAsync(d, h->d, sizeof(float) * h->n, cudaMemcpyDeviceToDevice, st);
    return lb_check("l-BFGS direction");
}

extern "C" int efwi_lbfgs_iterate(efwi_lbfgs *h, float *x, double *phi, float *g, efwi_objective_fn fn, void *ctx,
                                  efwi_lbfgs_info_t *info, efwi_stream_t stream) {
    if (!h || !x || !phi || !g || !fn || !info) return lb_fail(EFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = h->n;
    const int G = lb_grid(n);
    double *tmp = h->dev + h->o_tmp();
    *info = efwi_lbfgs_info_t{};
    info->phi_prev = *phi;
    info->phi = *phi;
    Search ls{h, x, fn, ctx, st};
    ls.phi0 = *phi;
    for (int attempt = 0; attempt < 2; ++attempt) {
        lb_direction(h, g, st);
        dot_dev(h, g, h->d, tmp, 1.0, nullptr, st);
        if (read_scalar(tmp, &ls.dphi0, st) != EFWI_OK) return lb_fail(EFWI_ERR_CUDA, "l-BFGS: reading g^T d failed");
        if (ls.dphi0 < 0) break;
        h->order.clear();                       // not a descent direction: restart from -g
    }
    info->pairs = (int)h->order.size();
    if (!(ls.dphi0 < 0)) {
        info->ls_failed = 1;
        return lb_check("l-BFGS");
    }
    double a0 = 1.0;
    if (h->order.empty()) {                     // first step (or restart): unit length along d = -H_0 g
        dot_dev(h, h->d, h->d, tmp, 1.0, nullptr, st);
        double dd = 0;
        if (read_scalar(tmp, &dd, st) != EFWI_OK) return lb_fail(EFWI_ERR_CUDA, "l-BFGS: reading d^T d failed");
        a0 = h->step0 > 0 ? h->step0 / std::sqrt(dd) : std::fmin(1.0, 1.0 / std::sqrt(dd));
    }
    Trial t;
    const bool found = ls.run(a0, t);
    info->evals = ls.evals;
    if (ls.rc != EFWI_OK) return ls.rc;
    if (!found) {
        info->ls_failed = 1;
        return lb_check("l-BFGS line search");
    }
    // new pair s = x_t - x, y = g_t - g, then x = x_t, g = g_t
    const int k = h->free_slot();
    k_sub<<<G, kLbThreads, 0, st>>>(slot_s(h, k), h->xt, x, n);
    k_sub<<<G, kLbThreads, 0, st>>>(slot_y(h, k), h->gt, g, n);
    int acc = 0;
    const int rc = lb_accept_pair(h, k, st, &acc);
    if (rc != EFWI_OK) return rc;
    cudaMemcpyAsync(x, h->xt, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(g, h->gt, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
    info->alpha = t.a;
    info->phi = t.phi;
    info->rate = (*phi - t.phi) / *phi;         // eq. 13
    info->pairs = (int)h->order.size();
    *phi = t.phi;
    return lb_check("l-BFGS iterate");
}

extern "C" int efwi_lbfgs_run(efwi_lbfgs *h, float *x, float *g, efwi_objective_fn fn, void *ctx, int max_iter,
                              double min_rate, efwi_lbfgs_info_t *info, efwi_stream_t stream) {
    if (!h || !x || !g || !fn || !info) return lb_fail(EFWI_ERR_ARG, "NULL argument");
    if (max_iter < 0) return lb_fail(EFWI_ERR_ARG, "max_iter must be >= 0");
    double phi = 0;
    const int r = fn(ctx, x, &phi, g, stream);
    if (r != 0) return lb_fail(r < 0 ? r : EFWI_ERR_ARG, "l-BFGS: the objective callback returned " + std::to_string(r));
    efwi_lbfgs_info_t it{};
    it.phi = it.phi_prev = phi;
    int evals = 1, k = 0, stop = EFWI_LBFGS_STOP_MAX_ITER;
    for (; k < max_iter; ++k) {
        const int rc = efwi_lbfgs_iterate(h, x, &phi, g, fn, ctx, &it, stream);
        evals += it.evals;
        if (rc != EFWI_OK) return rc;
        if (it.ls_failed) {
            stop = EFWI_LBFGS_STOP_NO_STEP;
            break;
        }
        if (it.rate < min_rate) {               // eq. 13 below the threshold
            stop = EFWI_LBFGS_STOP_RATE;
            ++k;
            break;
        }
    }
    it.iters = k;
    it.evals = evals;
    it.stop = stop;
    *info = it;
    return EFWI_OK;
}

// ---------------------------------------------------------------------------
// One iteration with the line search on the device.  Before the search the
// host computes the direction and reads g^T d (restart from -g when it is not a
// descent direction) and, on a first step, d^T d; the search itself is one
// launch of a graph whose conditional while-node repeats trial point,
// objective, phi' and search step; after it one read of the search state, then
// the pair update of efwi_lbfgs_iterate.
// ---------------------------------------------------------------------------
extern "C" int efwi_lbfgs_iterate_device(efwi_lbfgs *h, float *x, double *phi, float *g,
                                         efwi_device_objective_fn fn, void *ctx, efwi_lbfgs_info_t *info,
                                         efwi_stream_t stream) {
    if (!h || !x || !phi || !g || !fn || !info) return lb_fail(EFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = h->n;
    const int G = lb_grid(n);
    double *tmp = h->dev + h->o_tmp();
    if (!h->ls_state) {
        if (cudaMalloc(&h->ls_state, sizeof(LsState)) != cudaSuccess ||
            cudaMalloc((void **)&h->ls_phit, 2 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return lb_fail(EFWI_ERR_OOM, "l-BFGS: allocation of the device line-search state failed");
        }
        cudaStreamCreateWithFlags(&h->ls_cap, cudaStreamNonBlocking);
    }
    LsState *state = static_cast<LsState *>(h->ls_state);
    double *phit = h->ls_phit, *dphit = h->ls_phit + 1;
    *info = efwi_lbfgs_info_t{};
    double phi0 = 0;
    if (read_scalar(phi, &phi0, st) != EFWI_OK) return lb_fail(EFWI_ERR_CUDA, "l-BFGS: reading phi failed");
    info->phi_prev = info->phi = phi0;
    double dphi0 = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        lb_direction(h, g, st);
        dot_dev(h, g, h->d, tmp, 1.0, nullptr, st);
        if (read_scalar(tmp, &dphi0, st) != EFWI_OK) return lb_fail(EFWI_ERR_CUDA, "l-BFGS: reading g^T d failed");
        if (dphi0 < 0) break;
        h->order.clear();                       // not a descent direction: restart from -g
    }
    info->pairs = (int)h->order.size();
    if (!(dphi0 < 0)) {
        info->ls_failed = 1;
        return lb_check("l-BFGS");
    }
    double a0 = 1.0;
    if (h->order.empty()) {                     // first step (or restart): unit length along d = -H_0 g
        double dd = 0;
        dot_dev(h, h->d, h->d, tmp, 1.0, nullptr, st);
        if (read_scalar(tmp, &dd, st) != EFWI_OK) return lb_fail(EFWI_ERR_CUDA, "l-BFGS: reading d^T d failed");
        a0 = h->step0 > 0 ? h->step0 / std::sqrt(dd) : std::fmin(1.0, 1.0 / std::sqrt(dd));
    }
    // the search graph of this objective and these arrays (captured once, then replayed)
    const void *key[5] = {(const void *)fn, ctx, x, phi, g};
    bool same = h->ls_exec != nullptr;
    for (int k = 0; k < 5; ++k) same = same && key[k] == h->ls_key[k];
    if (!same) {
        cudaStreamSynchronize(st);
        lb_drop_graph(h);
        cudaGraph_t graph = nullptr;
        if (cudaGraphCreate(&graph, 0) != cudaSuccess) return lb_check("l-BFGS: graph creation");
        cudaGraphConditionalHandle cond;
        cudaGraphNodeParams np{};
        cudaGraphNode_t node;
        if (cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return lb_check("l-BFGS: conditional handle");
        }
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return lb_check("l-BFGS: conditional node");
        }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(h->ls_cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess) {
            cudaGraphDestroy(graph);
            return lb_check("l-BFGS: capture of the search body");
        }
        k_trial_state<<<G, kLbThreads, 0, h->ls_cap>>>(h->xt, x, h->d, n, state);
        const int r = fn(ctx, h->xt, phit, h->gt, (efwi_stream_t)h->ls_cap);
        dot_dev(h, h->gt, h->d, dphit, 1.0, nullptr, h->ls_cap);
        k_ls_step<<<1, 1, 0, h->ls_cap>>>(state, phit, dphit, cond);
        cudaGraph_t captured = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(h->ls_cap, &captured);
        if (r != 0 || ec != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(graph);
            if (r != 0) return lb_fail(r < 0 ? r : EFWI_ERR_ARG, "l-BFGS: the objective returned " + std::to_string(r) +
                                                                     " while its evaluation was captured");
            return lb_fail(EFWI_ERR_CUDA, std::string("l-BFGS: capture of the search body: ") + cudaGetErrorString(ec));
        }
        const cudaError_t ei = cudaGraphInstantiate(&h->ls_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            h->ls_exec = nullptr;
            return lb_fail(EFWI_ERR_CUDA, std::string("l-BFGS: instantiation of the search graph: ") +
                                              cudaGetErrorString(ei));
        }
        for (int k = 0; k < 5; ++k) h->ls_key[k] = key[k];
    }
    k_ls_init<<<1, 1, 0, st>>>(state, phi0, dphi0, a0, h->c1, h->c2, h->max_ls);
    if (cudaGraphLaunch(h->ls_exec, st) != cudaSuccess) return lb_check("l-BFGS: search graph launch");
    LsState s;
    if (cudaMemcpyAsync(&s, state, sizeof(LsState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return lb_fail(EFWI_ERR_CUDA, "l-BFGS: reading the search state failed");
    info->evals = s.evals;
    if (!s.ok) {
        info->ls_failed = 1;
        return lb_check("l-BFGS line search");
    }
    // the accepted step is the last trial: its point and gradient are in xt, gt
    const int k = h->free_slot();
    k_sub<<<G, kLbThreads, 0, st>>>(slot_s(h, k), h->xt, x, n);
    k_sub<<<G, kLbThreads, 0, st>>>(slot_y(h, k), h->gt, g, n);
    int acc = 0;
    const int rc = lb_accept_pair(h, k, st, &acc);
    if (rc != EFWI_OK) return rc;
    cudaMemcpyAsync(x, h->xt, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(g, h->gt, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(phi, phit, sizeof(double), cudaMemcpyDeviceToDevice, st);
    info->alpha = s.out.a;
    info->phi = s.out.phi;
    info->rate = (phi0 - s.out.phi) / phi0;     // eq. 13
    info->pairs = (int)h->order.size();
    return lb_check("l-BFGS iterate (device search)");
}
