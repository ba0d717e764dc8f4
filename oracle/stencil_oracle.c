/*
 * FP64 stencil oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow double-precision statement of what the stencil library computes (one thread,
 * or its cell loops split over host threads when built with OpenMP; the bits are the same).
 * Only the test suite, the package's smoke check and the benchmark's CPU-baseline leg load
 * it; the library never does, and this file shares no header, table or helper with the CUDA
 * path.  Every loop visits cells in row-major order (last axis fastest) and sums the
 * offsets of a stencil in canonical order, one term at a time, starting from 0.0.  Build with
 * -ffp-contract=off so that no multiply-add is fused and the results are identical on every
 * host.
 *
 * Sources (ForgeStencil paper):
 *   Sec. 2.1 (background, "Stencils, their variety, and the bandwidth limit"): the update
 *     u^{t+1}(x) = sum_{delta in S} c_delta u^t(x + delta), offset set S, star and box types,
 *     order r = max ||delta||_inf, variable coefficients as one more array per offset,
 *     storage precision f16/f32/f64.
 *   Sec. 4.3: temporal blocking ("diamond" family) fuses several time steps; the fused result
 *     equals the same number of single sweeps.
 * Readings where the paper is silent (stated again beside each function):
 *   - canonical offset order: lexicographic in (dz, dy, dx), each from -r to r;
 *   - diamond: the L1 ball ||delta||_1 <= r;
 *   - zero Dirichlet: every cell is updated, reads outside the grid return 0;
 *   - periodic: reads wrap, b(i) = i mod n;
 *   - div(k grad u): conservative 7-point (2D: 5-point) form, face k = arithmetic mean, k
 *     clamped (ghost k = k_p) and u zero outside a Dirichlet grid;
 *   - adjoint: the transpose of the linear map above;
 *   - low-precision storage: round to nearest, ties to even, after every step;
 *   - the acoustic wave equation, its misfit and its adjoint velocity gradient are not in the
 *     paper; they are written from the discretisation itself (leapfrog, Laplacian as above).
 * Parity pins for every function live in the CPU test suite (closed forms, FFT, brute force,
 * dot tests, finite differences).  Nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Built twice from this file: without OpenMP (one thread), and with -fopenmp, where the cell
 * loops below are split over threads.  Every cell is written by one thread and its terms are
 * summed in the same order either way, so both builds give the same bits. */
#ifdef _OPENMP
#include <omp.h>
#define PARALLEL_CELLS _Pragma("omp parallel for schedule(static)")
#else
#define PARALLEL_CELLS
#endif

/* Threads the cell loops use from now on (n <= 0: every host core); returns the count in
 * effect, 1 for the build without OpenMP. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n <= 0)
        n = omp_get_num_procs();
    omp_set_num_threads(n);
    return n;
#else
    (void)n;
    return 1;
#endif
}

#define ORC_STAR 0
#define ORC_BOX 1
#define ORC_DIAMOND 2

#define ORC_DIRICHLET0 0
#define ORC_PERIODIC 1

#define ORC_ROUND_NONE 0
#define ORC_ROUND_F32 1
#define ORC_ROUND_F16 2
#define ORC_ROUND_BF16 3

/* ------------------------------------------------------------------------------------------
 * Offset sets (Sec. 2.1).  Components are written slowest axis first: (dz, dy, dx) in 3D,
 * (dy, dx) in 2D.  Returns the number of offsets; `out` (if not NULL) receives n*ndim ints.
 * ---------------------------------------------------------------------------------------- */
int64_t orc_offsets(int ndim, int shape, int r, int32_t *out)
{
    if (ndim < 1 || ndim > 3 || r < 0)
        return -1;
    int64_t total = 1;
    for (int k = 0; k < ndim; ++k)
        total *= (2 * r + 1);
    int64_t n = 0;
    for (int64_t code = 0; code < total; ++code) {
        /* decode `code` as ndim base-(2r+1) digits, most significant digit = slowest axis */
        int d[3];
        int64_t c = code;
        for (int k = ndim - 1; k >= 0; --k) {
            d[k] = (int)(c % (2 * r + 1)) - r;
            c /= (2 * r + 1);
        }
        int nonzero = 0, l1 = 0;
        for (int k = 0; k < ndim; ++k) {
            if (d[k] != 0)
                nonzero++;
            l1 += abs(d[k]);
        }
        int keep;
        if (shape == ORC_STAR)
            keep = (nonzero <= 1);
        else if (shape == ORC_BOX)
            keep = 1;
        else if (shape == ORC_DIAMOND)
            keep = (l1 <= r);
        else
            return -1;
        if (!keep)
            continue;
        if (out)
            for (int k = 0; k < ndim; ++k)
                out[n * ndim + k] = d[k];
        n++;
    }
    return n;
}

/* ------------------------------------------------------------------------------------------
 * Index helpers.
 * ---------------------------------------------------------------------------------------- */
static int64_t wrap_index(int64_t i, int64_t n)
{
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

/* Multi-index of linear cell index `lin` (row-major, last axis fastest). */
static void unravel(int ndim, const int64_t *dims, int64_t lin, int64_t *p)
{
    for (int k = ndim - 1; k >= 0; --k) {
        p[k] = lin % dims[k];
        lin /= dims[k];
    }
}

/* Linear index of p + sign*d under the boundary rule; returns 0 if the read falls outside a
 * Dirichlet grid (the caller then uses the value 0). */
static int shifted_index(int ndim, const int64_t *dims, const int64_t *p, const int32_t *d,
                         int sign, int bc, int64_t *lin)
{
    int64_t acc = 0;
    for (int k = 0; k < ndim; ++k) {
        int64_t q = p[k] + (int64_t)sign * d[k];
        if (q < 0 || q >= dims[k]) {
            if (bc == ORC_PERIODIC)
                q = wrap_index(q, dims[k]);
            else
                return 0;
        }
        acc = acc * dims[k] + q;
    }
    *lin = acc;
    return 1;
}

static int64_t cell_count(int ndim, const int64_t *dims)
{
    int64_t n = 1;
    for (int k = 0; k < ndim; ++k)
        n *= dims[k];
    return n;
}

/* ------------------------------------------------------------------------------------------
 * One sweep, constant coefficients: out[p] = sum_o c[o] * in[b(p + off_o)]  (Sec. 2.1).
 * ---------------------------------------------------------------------------------------- */
void orc_sweep_const(int ndim, const int64_t *dims, int64_t npts, const int32_t *offs,
                     const double *c, int bc, const double *in, double *out)
{
    int64_t ncell = cell_count(ndim, dims);
    PARALLEL_CELLS
    for (int64_t lin = 0; lin < ncell; ++lin) {
        int64_t p[3];
        unravel(ndim, dims, lin, p);
        double acc = 0.0;
        for (int64_t o = 0; o < npts; ++o) {
            int64_t q;
            if (shifted_index(ndim, dims, p, offs + o * ndim, +1, bc, &q))
                acc += c[o] * in[q];
        }
        out[lin] = acc;
    }
}

/* The same sweep evaluated only at the listed cells (linear indices), for spot checks of
 * grids too large to sweep here. */
void orc_sweep_const_points(int ndim, const int64_t *dims, int64_t npts, const int32_t *offs,
                            const double *c, int bc, const double *in, int64_t nsel,
                            const int64_t *sel, double *out)
{
    PARALLEL_CELLS
    for (int64_t s = 0; s < nsel; ++s) {
        int64_t p[3];
        unravel(ndim, dims, sel[s], p);
        double acc = 0.0;
        for (int64_t o = 0; o < npts; ++o) {
            int64_t q;
            if (shifted_index(ndim, dims, p, offs + o * ndim, +1, bc, &q))
                acc += c[o] * in[q];
        }
        out[s] = acc;
    }
}

/* ------------------------------------------------------------------------------------------
 * One sweep, variable coefficients (Sec. 2.1: coefficients that vary in space are arrays):
 *   out[p] = sum_o w[o][p] * in[b(p + off_o)],   w stored as npts arrays of ncell values.
 * ---------------------------------------------------------------------------------------- */
void orc_sweep_var(int ndim, const int64_t *dims, int64_t npts, const int32_t *offs,
                   const double *w, int bc, const double *in, double *out)
{
    int64_t ncell = cell_count(ndim, dims);
    PARALLEL_CELLS
    for (int64_t lin = 0; lin < ncell; ++lin) {
        int64_t p[3];
        unravel(ndim, dims, lin, p);
        double acc = 0.0;
        for (int64_t o = 0; o < npts; ++o) {
            int64_t q;
            if (shifted_index(ndim, dims, p, offs + o * ndim, +1, bc, &q))
                acc += w[o * ncell + lin] * in[q];
        }
        out[lin] = acc;
    }
}

/* ------------------------------------------------------------------------------------------
 * Adjoint (transpose) of the sweeps above.  The forward map has entries A[p][b(p+o)] += w_o[p];
 * its transpose applied to y is (A^T y)[q] = sum_o w_o[b(q-o)] * y[b(q-o)], the terms whose
 * source cell q-o lies outside a Dirichlet grid being absent.
 * ---------------------------------------------------------------------------------------- */
void orc_sweep_const_adjoint(int ndim, const int64_t *dims, int64_t npts, const int32_t *offs,
                             const double *c, int bc, const double *y, double *out)
{
    int64_t ncell = cell_count(ndim, dims);
    PARALLEL_CELLS
    for (int64_t lin = 0; lin < ncell; ++lin) {
        int64_t q[3];
        unravel(ndim, dims, lin, q);
        double acc = 0.0;
        for (int64_t o = 0; o < npts; ++o) {
            int64_t src;
            if (shifted_index(ndim, dims, q, offs + o * ndim, -1, bc, &src))
                acc += c[o] * y[src];
        }
        out[lin] = acc;
    }
}

void orc_sweep_var_adjoint(int ndim, const int64_t *dims, int64_t npts, const int32_t *offs,
                           const double *w, int bc, const double *y, double *out)
{
    int64_t ncell = cell_count(ndim, dims);
    PARALLEL_CELLS
    for (int64_t lin = 0; lin < ncell; ++lin) {
        int64_t q[3];
        unravel(ndim, dims, lin, q);
        double acc = 0.0;
        for (int64_t o = 0; o < npts; ++o) {
            int64_t src;
            if (shifted_index(ndim, dims, q, offs + o * ndim, -1, bc, &src))
                acc += w[o * ncell + src] * y[src];
        }
        out[lin] = acc;
    }
}

/* ------------------------------------------------------------------------------------------
 * div(k grad u) with unit spacing, conservative form (a variable-coefficient stencil of
 * Sec. 2.1; the discretisation is this library's reading):
 *   out[p] = sum_axes [ kf+ (u[p+e] - u[p]) - kf- (u[p] - u[p-e]) ],
 *   kf+- = (k[p] + k[p+-e]) / 2.
 * Dirichlet: u outside the grid is 0 and k outside is k[p] (so a boundary face carries k[p]).
 * Periodic: both wrap.
 * ---------------------------------------------------------------------------------------- */
static void divk_faces(int ndim, const int64_t *dims, const int64_t *p, int axis, int bc,
                       const double *k, const double *u, int64_t lin, double *kf_plus,
                       double *kf_minus, double *u_plus, double *u_minus)
{
    int32_t e[3] = {0, 0, 0};
    e[axis] = 1;
    int64_t q;
    if (shifted_index(ndim, dims, p, e, +1, bc, &q)) {
        *kf_plus = 0.5 * (k[lin] + k[q]);
        *u_plus = u[q];
    } else {
        *kf_plus = 0.5 * (k[lin] + k[lin]);
        *u_plus = 0.0;
    }
    if (shifted_index(ndim, dims, p, e, -1, bc, &q)) {
        *kf_minus = 0.5 * (k[lin] + k[q]);
        *u_minus = u[q];
    } else {
        *kf_minus = 0.5 * (k[lin] + k[lin]);
        *u_minus = 0.0;
    }
}

void orc_divkgrad(int ndim, const int64_t *dims, const double *k, int bc, const double *u,
                  double *out)
{
    int64_t ncell = cell_count(ndim, dims);
    PARALLEL_CELLS
    for (int64_t lin = 0; lin < ncell; ++lin) {
        int64_t p[3];
        unravel(ndim, dims, lin, p);
        double acc = 0.0;
        for (int axis = 0; axis < ndim; ++axis) {
            double kp, km, up, um;
            divk_faces(ndim, dims, p, axis, bc, k, u, lin, &kp, &km, &up, &um);
            acc += kp * (up - u[lin]) - km * (u[lin] - um);
        }
        out[lin] = acc;
    }
}

/* The same operator written as per-offset coefficient arrays over the star-1 offsets in
 * canonical order (w_{+-e}[p] = kf+-, w_0[p] = -(sum of the 2*ndim faces)).  Writes
 * (2*ndim+1) * ncell doubles. */
void orc_divkgrad_weights(int ndim, const int64_t *dims, const double *k, int bc, double *w)
{
    int64_t ncell = cell_count(ndim, dims);
    int32_t offs[7 * 3];
    int64_t npts = orc_offsets(ndim, ORC_STAR, 1, offs);
    PARALLEL_CELLS
    for (int64_t lin = 0; lin < ncell; ++lin) {
        int64_t p[3];
        unravel(ndim, dims, lin, p);
        double centre = 0.0;
        for (int64_t o = 0; o < npts; ++o)
            w[o * ncell + lin] = 0.0;
        for (int axis = 0; axis < ndim; ++axis) {
            int32_t e[3] = {0, 0, 0};
            e[axis] = 1;
            int64_t q;
            double kp, km;
            if (shifted_index(ndim, dims, p, e, +1, bc, &q))
                kp = 0.5 * (k[lin] + k[q]);
            else
                kp = 0.5 * (k[lin] + k[lin]);
            if (shifted_index(ndim, dims, p, e, -1, bc, &q))
                km = 0.5 * (k[lin] + k[q]);
            else
                km = 0.5 * (k[lin] + k[lin]);
            for (int64_t o = 0; o < npts; ++o) {
                const int32_t *d = offs + o * ndim;
                int match_plus = 1, match_minus = 1;
                for (int a = 0; a < ndim; ++a) {
                    if (d[a] != (a == axis ? 1 : 0))
                        match_plus = 0;
                    if (d[a] != (a == axis ? -1 : 0))
                        match_minus = 0;
                }
                if (match_plus)
                    w[o * ncell + lin] = kp;
                if (match_minus)
                    w[o * ncell + lin] = km;
            }
            centre -= kp + km;
        }
        for (int64_t o = 0; o < npts; ++o) {
            const int32_t *d = offs + o * ndim;
            int zero = 1;
            for (int a = 0; a < ndim; ++a)
                if (d[a] != 0)
                    zero = 0;
            if (zero)
                w[o * ncell + lin] = centre;
        }
    }
}

/* ------------------------------------------------------------------------------------------
 * Rounding to a storage format, round-to-nearest with ties to even, written from the IEEE 754
 * definition of a binary format with `prec` significand bits (implicit bit included) and
 * exponent range [emin, emax]:  binary16 (11, -14, 15), bfloat16 (8, -126, 127),
 * binary32 (24, -126, 127).  Values beyond the largest finite number by half an ulp or more
 * become infinities.
 * ---------------------------------------------------------------------------------------- */
static double round_to_format(double x, int prec, int emin, int emax)
{
    if (x == 0.0 || !isfinite(x))
        return x;
    int e2;
    (void)frexp(x, &e2);  /* |x| = m * 2^e2, m in [0.5, 1): leading bit has weight 2^(e2-1) */
    int lead = e2 - 1;
    if (lead < emin)
        lead = emin;       /* subnormal range: fixed quantum */
    int q = lead - (prec - 1); /* quantum 2^q */
    double scaled = ldexp(x, -q);
    double fl = floor(scaled);
    double frac = scaled - fl;
    double r;
    if (frac > 0.5)
        r = fl + 1.0;
    else if (frac < 0.5)
        r = fl;
    else
        r = (fmod(fl, 2.0) == 0.0) ? fl : fl + 1.0;
    double y = ldexp(r, q);
    double maxfinite = ldexp(2.0 - ldexp(1.0, 1 - prec), emax);
    if (fabs(y) > maxfinite)
        return x > 0 ? INFINITY : -INFINITY;
    return y;
}

double orc_round_scalar(double x, int mode)
{
    switch (mode) {
    case ORC_ROUND_F32:
        return round_to_format(x, 24, -126, 127);
    case ORC_ROUND_F16:
        return round_to_format(x, 11, -14, 15);
    case ORC_ROUND_BF16:
        return round_to_format(x, 8, -126, 127);
    default:
        return x;
    }
}

void orc_round(int64_t n, double *x, int mode)
{
    if (mode == ORC_ROUND_NONE)
        return;
    PARALLEL_CELLS
    for (int64_t i = 0; i < n; ++i)
        x[i] = orc_round_scalar(x[i], mode);
}

/* ------------------------------------------------------------------------------------------
 * Several time steps: u^{t+1} = A u^t, iterated `steps` times (Sec. 2.1), with the optional
 * rounding to the storage format after every step (a fused multi-step sweep has the same
 * semantics as that many single sweeps, Sec. 4.3).  kind: 0 const, 1 var, 2 div(k grad u);
 * adjoint != 0 applies A^T instead.  `in` is not modified; `out` receives u^steps.
 * ---------------------------------------------------------------------------------------- */
int orc_run(int ndim, const int64_t *dims, int kind, int adjoint, int64_t npts,
            const int32_t *offs, const double *coef, int bc, int steps, int round_mode,
            const double *in, double *out)
{
    int64_t ncell = cell_count(ndim, dims);
    double *a = (double *)malloc(sizeof(double) * ncell);
    double *b = (double *)malloc(sizeof(double) * ncell);
    if (!a || !b) {
        free(a);
        free(b);
        return -1;
    }
    memcpy(a, in, sizeof(double) * ncell);
    for (int s = 0; s < steps; ++s) {
        if (kind == 0 && !adjoint)
            orc_sweep_const(ndim, dims, npts, offs, coef, bc, a, b);
        else if (kind == 0)
            orc_sweep_const_adjoint(ndim, dims, npts, offs, coef, bc, a, b);
        else if (kind == 1 && !adjoint)
            orc_sweep_var(ndim, dims, npts, offs, coef, bc, a, b);
        else if (kind == 1)
            orc_sweep_var_adjoint(ndim, dims, npts, offs, coef, bc, a, b);
        else if (kind == 2) {
            if (!adjoint) {
                orc_divkgrad(ndim, dims, coef, bc, a, b);
            } else {
                /* the transpose of div(k grad u), from its explicit coefficient arrays */
                int64_t n7 = 2 * ndim + 1;
                int32_t o7[7 * 3];
                orc_offsets(ndim, ORC_STAR, 1, o7);
                double *w = (double *)malloc(sizeof(double) * n7 * ncell);
                if (!w) {
                    free(a);
                    free(b);
                    return -1;
                }
                orc_divkgrad_weights(ndim, dims, coef, bc, w);
                orc_sweep_var_adjoint(ndim, dims, n7, o7, w, bc, a, b);
                free(w);
            }
        } else {
            free(a);
            free(b);
            return -2;
        }
        orc_round(ncell, b, round_mode);
        double *t = a;
        a = b;
        b = t;
    }
    memcpy(out, a, sizeof(double) * ncell);
    free(a);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Reaction-diffusion steps: a stencil fused with pointwise physics (Sec. 4.3 fuses a stencil
 * with an application's physics into one kernel; the equation is this library's example):
 *   u^{t+1} = u^t + dt * ( (A u^t) + c1 u^t + c3 (u^t)^3 ),
 * A the constant-coefficient sweep above, every term in FP64, the result rounded to the
 * storage format after each step.  `in` is not modified; `out` receives u^steps.
 * ---------------------------------------------------------------------------------------- */
int orc_reaction_run(int ndim, const int64_t *dims, int64_t npts, const int32_t *offs,
                     const double *c, int bc, int steps, double dt, double c1, double c3,
                     int round_mode, const double *in, double *out)
{
    int64_t ncell = cell_count(ndim, dims);
    double *a = (double *)malloc(sizeof(double) * ncell);
    double *lap = (double *)malloc(sizeof(double) * ncell);
    if (!a || !lap) {
        free(a);
        free(lap);
        return -1;
    }
    memcpy(a, in, sizeof(double) * ncell);
    for (int t = 0; t < steps; ++t) {
        orc_sweep_const(ndim, dims, npts, offs, c, bc, a, lap);
        for (int64_t i = 0; i < ncell; ++i)
            a[i] = a[i] + dt * (lap[i] + c1 * a[i] + c3 * a[i] * a[i] * a[i]);
        orc_round(ncell, a, round_mode);
    }
    memcpy(out, a, sizeof(double) * ncell);
    free(a);
    free(lap);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Acoustic wave equation on a 3D grid (not in the paper; written from the discretisation).
 *   u^{-1} = u^0 = 0,
 *   u^{n+1} = 2 u^n - u^{n-1} + a (.) (L u^n) + dt^2 s(t_n) e_src,    n = 0 .. N-1,
 * with a = (v dt / h)^2, L the unit-spacing Laplacian given as a constant-coefficient star
 * (zero Dirichlet), s the source time function and e_src the unit vector at the source cell.
 * Receivers: every (y, x) of plane z = rz; trace[n-1][y][x] = u^n[rz][y][x] for n = 1 .. N.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int64_t dims[3];
    int64_t npts;
    const int32_t *offs;
    const double *c;
    double h, dt;
    int nsteps;
    int64_t src;   /* linear index of the source cell */
    const double *wavelet;
    int64_t rz;
} wave_problem;

static void wave_step(const wave_problem *P, const double *a, const double *u,
                      const double *u_prev, int n, double *u_next, double *lu)
{
    int64_t ncell = P->dims[0] * P->dims[1] * P->dims[2];
    orc_sweep_const(3, P->dims, P->npts, P->offs, P->c, ORC_DIRICHLET0, u, lu);
    for (int64_t i = 0; i < ncell; ++i)
        u_next[i] = 2.0 * u[i] - u_prev[i] + a[i] * lu[i];
    u_next[P->src] += P->dt * P->dt * P->wavelet[n];
}

static void record(const wave_problem *P, const double *u, double *trace_row)
{
    int64_t plane = P->dims[1] * P->dims[2];
    memcpy(trace_row, u + P->rz * plane, sizeof(double) * plane);
}

static void wave_a(const wave_problem *P, const double *v, double *a)
{
    int64_t ncell = P->dims[0] * P->dims[1] * P->dims[2];
    for (int64_t i = 0; i < ncell; ++i) {
        double s = v[i] * P->dt / P->h;
        a[i] = s * s;
    }
}

/* Forward run: writes the N receiver rows (N * ny * nx) and, if u_last != NULL, u^N. */
int orc_wave_forward(const int64_t *dims, int64_t npts, const int32_t *offs, const double *c,
                     const double *v, double h, double dt, int nsteps, int64_t src,
                     const double *wavelet, int64_t rz, double *traces, double *u_last)
{
    wave_problem P = {{dims[0], dims[1], dims[2]}, npts, offs, c, h, dt, nsteps, src, wavelet, rz};
    int64_t ncell = dims[0] * dims[1] * dims[2];
    int64_t plane = dims[1] * dims[2];
    double *a = (double *)calloc(ncell, sizeof(double));
    double *u0 = (double *)calloc(ncell, sizeof(double));
    double *u1 = (double *)calloc(ncell, sizeof(double));
    double *u2 = (double *)calloc(ncell, sizeof(double));
    double *lu = (double *)calloc(ncell, sizeof(double));
    if (!a || !u0 || !u1 || !u2 || !lu) {
        free(a); free(u0); free(u1); free(u2); free(lu);
        return -1;
    }
    wave_a(&P, v, a);
    /* u0 = u^{n-1}, u1 = u^n */
    for (int n = 0; n < nsteps; ++n) {
        wave_step(&P, a, u1, u0, n, u2, lu);
        record(&P, u2, traces + (int64_t)n * plane);
        double *t = u0;
        u0 = u1;
        u1 = u2;
        u2 = t;
    }
    if (u_last)
        memcpy(u_last, u1, sizeof(double) * ncell);
    free(a); free(u0); free(u1); free(u2); free(lu);
    return 0;
}

/* Misfit J = 1/2 sum_n sum_receivers (trace - observed)^2, summed in index order. */
double orc_misfit(int64_t n, const double *traces, const double *observed)
{
    double j = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = traces[i] - observed[i];
        j += 0.5 * d * d;
    }
    return j;
}

/* Velocity gradient of J by the exact discrete adjoint of the forward run above.
 * With F^{n+1} = u^{n+1} - 2u^n + u^{n-1} - A u^n - f^n (A = diag(a) L) and
 * r^m = R^T (trace^m - observed^m), the multipliers satisfy, for m = N .. 1,
 *   lambda^m = r^m + 2 lambda^{m+1} + A^T lambda^{m+1} - lambda^{m+2},
 *   lambda^{N+1} = lambda^{N+2} = 0,   A^T y = L^T (a (.) y),
 * and dJ/da = sum_{m=1..N} lambda^m (.) L u^{m-1}, so g = dJ/dv = 2 v dt^2 / h^2 (.) dJ/da.
 * L^T is applied as the adjoint sweep (offset flipped, source cell q - o).
 * ck_every = 0 stores every u^n; otherwise (u^n, u^{n-1}) are kept at n = 0, k, 2k, ... and
 * each segment is recomputed from its checkpoint during the backward walk.  Both give the
 * same bits.  Returns J through *J_out. */
int orc_wave_gradient(const int64_t *dims, int64_t npts, const int32_t *offs, const double *c,
                      const double *v, double h, double dt, int nsteps, int64_t src,
                      const double *wavelet, int64_t rz, const double *observed,
                      int ck_every, double *g, double *J_out)
{
    wave_problem P = {{dims[0], dims[1], dims[2]}, npts, offs, c, h, dt, nsteps, src, wavelet, rz};
    int64_t ncell = dims[0] * dims[1] * dims[2];
    int64_t plane = dims[1] * dims[2];
    int N = nsteps;
    int k = ck_every > 0 ? ck_every : N;
    int nseg = (N + k - 1) / k;
    int store_all = (ck_every <= 0);
    /* storage: store-all keeps u^0..u^N; checkpointed keeps 2 fields per segment start plus a
     * segment buffer of k+1 fields. */
    int64_t nkeep = store_all ? (int64_t)(N + 1) : (int64_t)(2 * nseg + k + 1);
    double *keep = (double *)calloc((size_t)(nkeep * ncell), sizeof(double));
    double *a = (double *)calloc(ncell, sizeof(double));
    double *lu = (double *)calloc(ncell, sizeof(double));
    double *tmp = (double *)calloc(ncell, sizeof(double));
    double *lam0 = (double *)calloc(ncell, sizeof(double)); /* lambda^{m+2} */
    double *lam1 = (double *)calloc(ncell, sizeof(double)); /* lambda^{m+1} */
    double *lam2 = (double *)calloc(ncell, sizeof(double)); /* lambda^m     */
    double *traces = (double *)calloc((size_t)N * plane, sizeof(double));
    double *uprev = (double *)calloc(ncell, sizeof(double));
    double *ucur = (double *)calloc(ncell, sizeof(double));
    double *unext = (double *)calloc(ncell, sizeof(double));
    double *dJda = (double *)calloc(ncell, sizeof(double));
    if (!keep || !a || !lu || !tmp || !lam0 || !lam1 || !lam2 || !traces || !uprev || !ucur ||
        !unext || !dJda) {
        free(keep); free(a); free(lu); free(tmp); free(lam0); free(lam1); free(lam2);
        free(traces); free(uprev); free(ucur); free(unext); free(dJda);
        return -1;
    }
    wave_a(&P, v, a);

    /* forward sweep, recording traces and the kept states */
    double *ck = keep;                         /* checkpoint area (2 per segment) */
    double *seg = keep + (int64_t)2 * nseg * ncell; /* segment buffer (k+1 fields) */
    for (int n = 0; n <= N; ++n) {
        /* ucur = u^n, uprev = u^{n-1} here */
        if (store_all)
            memcpy(keep + (int64_t)n * ncell, ucur, sizeof(double) * ncell);
        else if (n % k == 0 && n < N) {
            int s = n / k;
            memcpy(ck + (int64_t)(2 * s) * ncell, ucur, sizeof(double) * ncell);
            memcpy(ck + (int64_t)(2 * s + 1) * ncell, uprev, sizeof(double) * ncell);
        }
        if (n == N)
            break;
        wave_step(&P, a, ucur, uprev, n, unext, lu);
        record(&P, unext, traces + (int64_t)n * plane);
        double *t = uprev;
        uprev = ucur;
        ucur = unext;
        unext = t;
    }
    double J = orc_misfit((int64_t)N * plane, traces, observed);

    /* backward walk over segments [n0, n1), newest first */
    for (int s = nseg - 1; s >= 0; --s) {
        int n0 = s * k;
        int n1 = n0 + k < N ? n0 + k : N;
        double *states; /* states[j] = u^{n0 + j}, j = 0 .. n1 - n0 - 1 */
        if (store_all) {
            states = keep + (int64_t)n0 * ncell;
        } else {
            states = seg;
            memcpy(ucur, ck + (int64_t)(2 * s) * ncell, sizeof(double) * ncell);
            memcpy(uprev, ck + (int64_t)(2 * s + 1) * ncell, sizeof(double) * ncell);
            for (int n = n0; n < n1; ++n) {
                memcpy(states + (int64_t)(n - n0) * ncell, ucur, sizeof(double) * ncell);
                if (n + 1 < n1) {
                    wave_step(&P, a, ucur, uprev, n, unext, lu);
                    double *t = uprev;
                    uprev = ucur;
                    ucur = unext;
                    unext = t;
                }
            }
        }
        for (int m = n1; m > n0; --m) {
            /* lam2 = lambda^m = r^m + 2 lambda^{m+1} + L^T (a (.) lambda^{m+1}) - lambda^{m+2} */
            for (int64_t i = 0; i < ncell; ++i)
                tmp[i] = a[i] * lam1[i];
            orc_sweep_const_adjoint(3, P.dims, npts, offs, c, ORC_DIRICHLET0, tmp, lu);
            for (int64_t i = 0; i < ncell; ++i)
                lam2[i] = 2.0 * lam1[i] + lu[i] - lam0[i];
            {
                const double *tr = traces + (int64_t)(m - 1) * plane;
                const double *ob = observed + (int64_t)(m - 1) * plane;
                double *row = lam2 + rz * plane;
                for (int64_t i = 0; i < plane; ++i)
                    row[i] += tr[i] - ob[i];
            }
            /* dJ/da += lambda^m (.) L u^{m-1} */
            orc_sweep_const(3, P.dims, npts, offs, c, ORC_DIRICHLET0,
                            states + (int64_t)(m - 1 - n0) * ncell, lu);
            for (int64_t i = 0; i < ncell; ++i)
                dJda[i] += lam2[i] * lu[i];
            double *t = lam0;
            lam0 = lam1;
            lam1 = lam2;
            lam2 = t;
        }
    }
    for (int64_t i = 0; i < ncell; ++i)
        g[i] = 2.0 * v[i] * dt * dt / (h * h) * dJda[i];
    if (J_out)
        *J_out = J;
    free(keep); free(a); free(lu); free(tmp); free(lam0); free(lam1); free(lam2);
    free(traces); free(uprev); free(ucur); free(unext); free(dJda);
    return 0;
}
