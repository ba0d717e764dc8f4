/*
 * GB300 stencil operator library -- acoustic wave equation driver (C ABI).
 *
 * A seismic application of the stencil sweep (ForgeStencil Sec. 2.1) and of its adjoint:
 * the 3D constant-density acoustic wave equation with a radius-r star Laplacian, advanced by
 * second-order leapfrog, its receiver misfit, and the velocity gradient of that misfit by the
 * exact discrete adjoint with checkpointing.  The paper reports no wave-equation results; the
 * discretisation below is this library's.
 *
 *   a = (v dt / h)^2,                         u^{-1} = u^0 = 0,
 *   u^{n+1} = 2 u^n - u^{n-1} + a (.) (L u^n) + dt^2 s_n e_src,      n = 0 .. N-1,
 *   L = sum_o c_o shift_o   (unit-spacing star weights c_o in canonical offset order, zero
 *                            Dirichlet ghosts),
 *   trace^n[y][x] = u^n[rz][y][x]            (receivers: the whole plane z = rz), n = 1 .. N,
 *   J = 1/2 sum_n sum_{y,x} (trace^n - observed^n)^2          (FP64),
 *   g = dJ/dv  (FP64), by the transposed leapfrog: lambda^m = r^m + 2 lambda^{m+1}
 *       + L^T (a (.) lambda^{m+1}) - lambda^{m+2},  g = 2 v dt^2 / h^2 (.) sum_m lambda^m (.)
 *       L u^{m-1}.  The device carries mu = a (.) lambda so each adjoint step is one sweep of
 *       the offset-flipped stencil; lambda = mu / a.
 *
 * Fields are f32; dims = (nz, ny, nx) slowest first; all array arguments are DEVICE pointers
 * owned by the caller; `stream` is a cudaStream_t as void*.  Return codes as in stencil.h.
 */
#ifndef GB300_WAVE_H
#define GB300_WAVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wave_plan_s *wave_handle;

/* wave_plan -- describe a run.
 *   dims[3]      grid (nz, ny, nx), each >= 2*radius+1.
 *   radius       star radius of the Laplacian (1, 2 or 4); lap[6*radius+1] its unit-spacing
 *                weights in canonical offset order (copied).
 *   h, dt        grid spacing and time step (dt is fixed: it is not differentiated).
 *   nsteps       N >= 1; wavelet[N] the source time function s_n (copied).
 *   src[3]       source cell (z, y, x); rz the receiver plane index.
 *   ck_every     checkpoint interval k >= 1 for wave_gradient (k >= N stores one segment).
 * Allocates no device memory (buffers are allocated on first use and kept by the plan). */
int wave_plan(wave_handle *out, const int64_t *dims, int radius, const double *lap, double h,
              double dt, int nsteps, const int64_t *src, const double *wavelet, int64_t rz,
              int ck_every);

/* wave_forward -- run the N steps for velocity v (dims) and write the receiver traces
 * (N x ny x nx, row n-1 = step n).  Asynchronous on `stream`. */
int wave_forward(wave_handle h, const float *v, float *traces, void *stream);

/* wave_misfit -- J = 1/2 sum (traces - observed)^2 over N x ny x nx values, in FP64 (fixed
 * summation order, so repeated calls give the same bits); writes one double to J (device). */
int wave_misfit(wave_handle h, const float *traces, const float *observed, double *J,
                void *stream);

/* wave_gradient -- forward run with checkpoints every ck_every steps, misfit J (one device
 * double) and gradient g (dims, FP64, device) against `observed` (N x ny x nx).  The backward
 * walk recomputes each segment from its checkpoint.  traces (N x ny x nx, device) receives the
 * forward traces.  Asynchronous on `stream`. */
int wave_gradient(wave_handle h, const float *v, const float *observed, float *traces,
                  double *J, double *g, void *stream);

/* wave_sync_status -- synchronise `stream` and return the first error latched by a step
 * kernel of this plan since the last call (STENCIL_ERR_TIMEOUT: a bounded device-side wait of
 * the plane ring expired and the step's output is incomplete), then clear it.  Read it with
 * the device that ran the plan current. */
int wave_sync_status(wave_handle h, void *stream);

/* wave_destroy -- free the plan and its device buffers (synchronises the device). */
int wave_destroy(wave_handle h);

#ifdef __cplusplus
}
#endif

#endif /* GB300_WAVE_H */
