// Acoustic wave equation: leapfrog forward step, adjoint step, FP64 misfit and gradient, and
// the checkpointed driver behind include/wave.h.
//
// Both steps run the streaming star kernel (the radius-R Laplacian L of a field with zero
// Dirichlet ghosts, tensor-copied plane by plane by a producer warp) with a fused epilogue
// that applies the rest of the update to each finished output:
//   forward:  u^{n+1} = 2u^n - u^{n-1} + a (.) L u^n (+ dt^2 s_n at the source cell),
//             optionally storing L u^n (segment recompute) and the receiver plane;
//   adjoint:  mu^m = 2mu^{m+1} - mu^{m+2} + a (.) L mu^{m+1} + a (.) r^m (receiver plane),
//             G += mu^m (.) L u^{m-1}  in FP64,
// where mu = a (.) lambda: the transposed operator L^T (a (.) lambda) = L mu (the radius-R
// Laplacian is symmetric), so each adjoint step is the flipped stencil applied to mu, and the
// velocity gradient is g = (2 / v) (.) G.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/stencil.h"
#include "../../include/wave.h"
#include "internal.h"
#include "stream_launch.cuh"
#include "var.cuh"

namespace gst {

// The fused update applied to each finished Laplacian row segment L (VY rows of 4 cells at
// (zo, oy, ox)) by the streaming star kernel, whose input `in` is the field under the stencil.
//   forward:  u^{n+1} = 2u^n - u^{n-1} + a (.) L u^n (+ dt^2 s_n at the source cell),
//             optionally storing L u^n and the receiver plane of u^{n+1};
//   adjoint:  mu^m = 2mu^{m+1} - mu^{m+2} + a (.) L mu^{m+1} (+ a (.) r^m on the receiver
//             plane), then G += mu^m (.) L u^{m-1} in FP64.
template <bool ADJ> struct WaveEpi {
    struct Params {
        const float *uprev;    // u^{n-1}, or mu^{m+2}
        const float *a;        // (v dt / h)^2
        float *unext;          // u^{n+1}, or mu^m
        float *lu_store;       // forward: L u^n (optional)
        float *trace_row;      // forward: receiver plane of u^{n+1} (optional)
        const float *res_t;    // adjoint: trace row of step m
        const float *res_o;    // adjoint: observed row of step m
        const float *lu_prev;  // adjoint: L u^{m-1}
        double *G;             // adjoint: sum of mu^m L u^{m-1}
        long long src;         // linear index of the source cell, -1 for none
        float src_val;         // dt^2 s_n
        int rz;                // receiver plane
    };
    // u^n (or mu^{m+1}) at the output, u^{n-1} (or mu^{m+2}), a, and for the adjoint L u^{m-1}
    template <int VY, int VX> struct Regs {
        float uc[VY][VX], up[VY][VX], av[VY][VX], lu[ADJ ? VY : 1][VX];
    };
    template <typename T, int VY, int VX>
    __device__ __forceinline__ static void prefetch(const StreamParams<T> &p, const Params &e,
                                                    int zo, int oy, int ox, bool vec,
                                                    int vy_valid, Regs<VY, VX> &r) {
        static_assert(sizeof(T) == 4, "the wave fields are f32");
        const int nx = p.nx, nvalid = nx - ox;
#pragma unroll
        for (int vy = 0; vy < VY; ++vy) {
            if (vy >= vy_valid) break;
            const size_t base = ((size_t)zo * p.ny + oy + vy) * nx + ox;
            load_cells<float, VX>(p.in + base, vec, nvalid, r.uc[vy]);
            load_cells<float, VX>(e.uprev + base, vec, nvalid, r.up[vy]);
            load_cells<float, VX>(e.a + base, vec, nvalid, r.av[vy]);
            if constexpr (ADJ) load_cells<float, VX>(e.lu_prev + base, vec, nvalid, r.lu[vy]);
        }
    }
    template <typename T, int VY, int VX>
    __device__ __forceinline__ static void apply(const StreamParams<T> &p, const Params &e,
                                                 int zo, int oy, int ox, bool vec, int vy_valid,
                                                 const Regs<VY, VX> &r,
                                                 const float (&L)[VY][VX]) {
        const int nx = p.nx, nvalid = nx - ox;
#pragma unroll
        for (int vy = 0; vy < VY; ++vy) {
            if (vy >= vy_valid) break;
            const size_t row = (size_t)(oy + vy) * nx + ox;
            const size_t base = (size_t)zo * nx * p.ny + row;
            float un[VX];
#pragma unroll
            for (int i = 0; i < VX; ++i)
                un[i] = fmaf(r.av[vy][i], L[vy][i], 2.0f * r.uc[vy][i] - r.up[vy][i]);
            if constexpr (!ADJ) {
                if (e.src >= 0 && (long long)base <= e.src && e.src < (long long)base + VX) {
#pragma unroll
                    for (int i = 0; i < VX; ++i)
                        if ((long long)base + i == e.src) un[i] += e.src_val;
                }
                store_cells<float, VX>(e.unext + base, vec, nvalid, un);
                if (e.lu_store) store_cells<float, VX>(e.lu_store + base, vec, nvalid, L[vy]);
                if (e.trace_row && zo == e.rz)
                    store_cells<float, VX>(e.trace_row + row, vec, nvalid, un);
            } else {
                if (zo == e.rz) {
                    float rt[VX], ro[VX];
                    load_cells<float, VX>(e.res_t + row, vec, nvalid, rt);
                    load_cells<float, VX>(e.res_o + row, vec, nvalid, ro);
#pragma unroll
                    for (int i = 0; i < VX; ++i) un[i] = fmaf(r.av[vy][i], rt[i] - ro[i], un[i]);
                }
                store_cells<float, VX>(e.unext + base, vec, nvalid, un);
#pragma unroll
                for (int i = 0; i < VX; ++i)
                    if (i < nvalid) e.G[base + i] += (double)un[i] * (double)r.lu[vy][i];
            }
        }
    }
};

__global__ void wave_a_kernel(const float *__restrict__ v, float *__restrict__ a, size_t n,
                              float dt_over_h) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float s = v[i] * dt_over_h;
        a[i] = s * s;
    }
}

__global__ void wave_grad_finish_kernel(const float *__restrict__ v, double *__restrict__ g,
                                        size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        g[i] = 2.0 / (double)v[i] * g[i];
}

// Misfit, pass 1: block b sums 1/2 (t - o)^2 over its contiguous chunk in index order, then a
// fixed tree; pass 2 sums the block partials in order.  Deterministic.
constexpr int kMisfitThreads = 256;
__global__ void misfit_partial_kernel(const float *__restrict__ t, const float *__restrict__ o,
                                      size_t n, size_t chunk, double *__restrict__ part) {
    __shared__ double red[kMisfitThreads];
    const size_t lo = blockIdx.x * chunk, hi = (lo + chunk < n) ? lo + chunk : n;
    double s = 0.0;
    for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double d = (double)t[i] - (double)o[i];
        s += 0.5 * d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kMisfitThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void misfit_final_kernel(const double *__restrict__ part, int nb, double *J) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += part[i];
        *J = s;
    }
}

}  // namespace gst

using namespace gst;

struct wave_plan_s {
    int64_t nz = 0, ny = 0, nx = 0;
    int radius = 0;
    std::vector<float> lap;
    double h = 1, dt = 1;
    int nsteps = 0;
    int64_t src = -1;
    std::vector<double> wavelet;
    int64_t rz = 0;
    int k = 1;
    // device buffers (allocated on first use)
    float *a = nullptr;
    float *w[3] = {nullptr, nullptr, nullptr};  // work fields
    float *mu[3] = {nullptr, nullptr, nullptr};
    std::vector<float *> ck;                     // 2 per segment: u^{n0}, u^{n0-1}
    std::vector<float *> seg;                    // k fields: L u^n within a segment
    double *part = nullptr;
    int nparts = 0;
    int status_slot = -1;   // device status word of the step kernels (status.cu)
    bool launched = false;
};

static size_t wave_cells(const wave_plan_s *p) { return (size_t)p->nz * p->ny * p->nx; }

static int walloc(float **ptr, size_t n) {
    if (*ptr) return STENCIL_OK;
    if (cudaMalloc(ptr, n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return STENCIL_ERR_OOM;
    }
    return STENCIL_OK;
}

static int wave_step(wave_plan_s *p, bool adj, const float *u, const float *uprev, float *unext,
                     float *lu_store, float *trace_row, const float *res_t, const float *res_o,
                     const float *lu_prev, double *G, long long src, float src_val,
                     cudaStream_t s) {
    typename WaveEpi<false>::Params e;  // same layout for both directions
    std::memset(&e, 0, sizeof(e));
    e.uprev = uprev;
    e.a = p->a;
    e.unext = unext;
    e.lu_store = lu_store;
    e.trace_row = trace_row;
    e.res_t = res_t;
    e.res_o = res_o;
    e.lu_prev = lu_prev;
    e.G = G;
    e.src = src;
    e.src_val = src_val;
    e.rz = (int)p->rz;
    StreamLaunch L;
    L.ndim = 3;
    L.nz = p->nz;
    L.ny = p->ny;
    L.nx = p->nx;
    L.shape = kStar;
    L.radius = p->radius;
    L.dtype = kF32;
    L.periodic = 0;
    L.coeffs = p->lap.data();
    L.in = u;
    L.out = unext;
    // measured on GB300 for the 256^3 radius-4 workload: 7 consumer rows per tile, 64-plane
    // z chunks, a 4-deep ring
    L.block_x = 32;
    L.block_y = 7;
    L.vec_y = 1;
    L.z_chunk = 64;
    L.stages = 4;
    L.err = status_word(p->status_slot);
    L.stream = s;
    p->launched = true;
    int rc;
    if (!adj) {
        const typename WaveEpi<false>::Params &ef = e;
        rc = p->radius == 1   ? launch_stream_t<float, 3, kStar, 1, 1, WaveEpi<false>>(L, ef)
             : p->radius == 2 ? launch_stream_t<float, 3, kStar, 2, 1, WaveEpi<false>>(L, ef)
                              : launch_stream_t<float, 3, kStar, 4, 1, WaveEpi<false>>(L, ef);
    } else {
        typename WaveEpi<true>::Params ea;
        static_assert(sizeof(ea) == sizeof(e), "one parameter layout");
        std::memcpy(&ea, &e, sizeof(e));
        rc = p->radius == 1   ? launch_stream_t<float, 3, kStar, 1, 1, WaveEpi<true>>(L, ea)
             : p->radius == 2 ? launch_stream_t<float, 3, kStar, 2, 1, WaveEpi<true>>(L, ea)
                              : launch_stream_t<float, 3, kStar, 4, 1, WaveEpi<true>>(L, ea);
    }
    return rc == 0 ? STENCIL_OK : (rc == -2 ? STENCIL_ERR_UNSUPPORTED : STENCIL_ERR_CUDA);
}

static int wave_compute_a(wave_plan_s *p, const float *v, cudaStream_t s) {
    int rc = walloc(&p->a, wave_cells(p));
    if (rc) return rc;
    wave_a_kernel<<<1024, 256, 0, s>>>(v, p->a, wave_cells(p), (float)(p->dt / p->h));
    count_launch();
    return cudaGetLastError() == cudaSuccess ? STENCIL_OK : STENCIL_ERR_CUDA;
}

// The forward run.  With `ck`, (u^n, u^{n-1}) are copied into the checkpoint buffers at every
// n = 0, k, 2k, ... < N before step n.
static int wave_run_forward(wave_plan_s *p, float *traces, bool checkpoints, cudaStream_t s) {
    const size_t n = wave_cells(p), plane = (size_t)p->ny * p->nx;
    for (int i = 0; i < 3; ++i) {
        int rc = walloc(&p->w[i], n);
        if (rc) return rc;
    }
    float *prev = p->w[0], *cur = p->w[1], *next = p->w[2];
    if (cudaMemsetAsync(prev, 0, n * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(cur, 0, n * sizeof(float), s) != cudaSuccess)
        return STENCIL_ERR_CUDA;
    for (int step = 0; step < p->nsteps; ++step) {
        if (checkpoints && step % p->k == 0) {
            const int sgi = step / p->k;
            if (cudaMemcpyAsync(p->ck[2 * sgi], cur, n * sizeof(float), cudaMemcpyDeviceToDevice,
                                s) != cudaSuccess ||
                cudaMemcpyAsync(p->ck[2 * sgi + 1], prev, n * sizeof(float),
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return STENCIL_ERR_CUDA;
        }
        const float sv = (float)(p->dt * p->dt * p->wavelet[step]);
        int rc = wave_step(p, false, cur, prev, next, nullptr, traces + (size_t)step * plane,
                           nullptr, nullptr, nullptr, nullptr, p->src, sv, s);
        if (rc) return rc;
        float *t = prev;
        prev = cur;
        cur = next;
        next = t;
    }
    return STENCIL_OK;
}

static int wave_misfit_impl(wave_plan_s *p, const float *t, const float *o, double *J,
                            cudaStream_t s) {
    const size_t n = (size_t)p->nsteps * p->ny * p->nx;
    const int nb = 1024;
    if (!p->part) {
        if (cudaMalloc(&p->part, nb * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return STENCIL_ERR_OOM;
        }
        p->nparts = nb;
    }
    const size_t chunk = (n + nb - 1) / nb;
    misfit_partial_kernel<<<nb, kMisfitThreads, 0, s>>>(t, o, n, chunk, p->part);
    misfit_final_kernel<<<1, 32, 0, s>>>(p->part, nb, J);
    count_launch(2);
    return cudaGetLastError() == cudaSuccess ? STENCIL_OK : STENCIL_ERR_CUDA;
}

extern "C" {

int wave_plan(wave_handle *out, const int64_t *dims, int radius, const double *lap, double h,
              double dt, int nsteps, const int64_t *src, const double *wavelet, int64_t rz,
              int ck_every) {
    if (!out) return STENCIL_ERR_BADARG;
    *out = nullptr;
    if (!dims || !lap || !src || !wavelet || nsteps < 1 || ck_every < 1) return STENCIL_ERR_BADARG;
    if (radius != 1 && radius != 2 && radius != 4) return STENCIL_ERR_UNSUPPORTED;
    if (!(h > 0) || !(dt > 0)) return STENCIL_ERR_BADARG;
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 2 * radius + 1 || src[i] < 0 || src[i] >= dims[i]) return STENCIL_ERR_BADARG;
    if (rz < 0 || rz >= dims[0]) return STENCIL_ERR_BADARG;
    if (dims[1] * dims[2] > ((int64_t)1 << 30) || dims[0] > ((int64_t)1 << 20))
        return STENCIL_ERR_UNSUPPORTED;
    wave_plan_s *p = new (std::nothrow) wave_plan_s();
    if (!p) return STENCIL_ERR_OOM;
    p->status_slot = status_acquire();
    if (p->status_slot < 0) {
        delete p;
        return STENCIL_ERR_OOM;
    }
    p->nz = dims[0];
    p->ny = dims[1];
    p->nx = dims[2];
    p->radius = radius;
    p->lap.assign(lap, lap + 6 * radius + 1);
    p->h = h;
    p->dt = dt;
    p->nsteps = nsteps;
    p->src = (src[0] * dims[1] + src[1]) * dims[2] + src[2];
    p->wavelet.assign(wavelet, wavelet + nsteps);
    p->rz = rz;
    p->k = std::min(ck_every, nsteps);
    *out = p;
    return STENCIL_OK;
}

int wave_forward(wave_handle h, const float *v, float *traces, void *stream) {
    if (!h || !v || !traces) return STENCIL_ERR_BADARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = wave_compute_a(h, v, s);
    if (rc) return rc;
    return wave_run_forward(h, traces, false, s);
}

int wave_misfit(wave_handle h, const float *traces, const float *observed, double *J,
                void *stream) {
    if (!h || !traces || !observed || !J) return STENCIL_ERR_BADARG;
    return wave_misfit_impl(h, traces, observed, J, (cudaStream_t)stream);
}

int wave_gradient(wave_handle h, const float *v, const float *observed, float *traces,
                  double *J, double *g, void *stream) {
    if (!h || !v || !observed || !traces || !J || !g) return STENCIL_ERR_BADARG;
    wave_plan_s *p = h;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = wave_cells(p), plane = (size_t)p->ny * p->nx;
    const int N = p->nsteps, k = p->k;
    const int nseg = (N + k - 1) / k;
    if ((int)p->ck.size() < 2 * nseg) p->ck.resize(2 * nseg, nullptr);
    if ((int)p->seg.size() < k) p->seg.resize(k, nullptr);
    for (int i = 0; i < 2 * nseg; ++i)
        if (walloc(&p->ck[i], n)) return STENCIL_ERR_OOM;
    for (int i = 0; i < k; ++i)
        if (walloc(&p->seg[i], n)) return STENCIL_ERR_OOM;
    for (int i = 0; i < 3; ++i)
        if (walloc(&p->mu[i], n)) return STENCIL_ERR_OOM;
    int rc = wave_compute_a(p, v, s);
    if (rc) return rc;
    rc = wave_run_forward(p, traces, true, s);
    if (rc) return rc;
    rc = wave_misfit_impl(p, traces, observed, J, s);
    if (rc) return rc;
    if (cudaMemsetAsync(g, 0, n * sizeof(double), s) != cudaSuccess) return STENCIL_ERR_CUDA;
    float *m0 = p->mu[0], *m1 = p->mu[1], *m2 = p->mu[2];  // mu^{m+2}, mu^{m+1}, mu^m
    if (cudaMemsetAsync(m0, 0, n * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(m1, 0, n * sizeof(float), s) != cudaSuccess)
        return STENCIL_ERR_CUDA;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int n0 = sg * k, n1 = std::min(n0 + k, N);
        // recompute u^{n0} .. u^{n1-1}, keeping L u^n for n in [n0, n1)
        const float *prev = p->ck[2 * sg + 1];
        const float *cur = p->ck[2 * sg];
        float *work[3] = {p->w[0], p->w[1], p->w[2]};
        int wi = 0;
        for (int step = n0; step < n1; ++step) {
            float *next = work[wi];
            wi = (wi + 1) % 3;
            const float sv = (float)(p->dt * p->dt * p->wavelet[step]);
            rc = wave_step(p, false, cur, prev, next, p->seg[step - n0], nullptr, nullptr,
                           nullptr, nullptr, nullptr, p->src, sv, s);
            if (rc) return rc;
            prev = cur;
            cur = next;
        }
        // adjoint steps m = n1 .. n0+1
        for (int m = n1; m > n0; --m) {
            rc = wave_step(p, true, m1, m0, m2, nullptr, nullptr,
                           traces + (size_t)(m - 1) * plane, observed + (size_t)(m - 1) * plane,
                           p->seg[m - 1 - n0], g, -1, 0.0f, s);
            if (rc) return rc;
            float *t = m0;
            m0 = m1;
            m1 = m2;
            m2 = t;
        }
    }
    wave_grad_finish_kernel<<<1024, 256, 0, s>>>(v, g, n);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? STENCIL_OK : STENCIL_ERR_CUDA;
}

int wave_sync_status(wave_handle h, void *stream) {
    if (!h) return STENCIL_ERR_BADARG;
    return status_take(h->status_slot, (cudaStream_t)stream);
}

int wave_destroy(wave_handle h) {
    if (!h) return STENCIL_OK;
    cudaDeviceSynchronize();
    status_release(h->status_slot, h->launched);
    cudaFree(h->a);
    for (int i = 0; i < 3; ++i) {
        cudaFree(h->w[i]);
        cudaFree(h->mu[i]);
    }
    for (float *q : h->ck) cudaFree(q);
    for (float *q : h->seg) cudaFree(q);
    cudaFree(h->part);
    delete h;
    return STENCIL_OK;
}

}  // extern "C"
