// A stencil fused with the pointwise physics of a reaction-diffusion equation (ForgeStencil
// Sec. 4.3: kernels that fuse a stencil with an application's physics into one launch).  One
// explicit step of
//     u^{t+1} = u^t + dt * ( (A u^t) + c1 u^t + c3 (u^t)^3 ),
// A the plan's constant-coefficient sweep (e.g. a diffusion Laplacian), c1 and c3 linear and
// cubic reaction rates (Allen-Cahn: c1 = 1/eps^2, c3 = -1/eps^2), runs as the streaming
// kernel with this epilogue: the stencil sum L = (A u)[p] of a finished output row segment
// and the cell's own value u[p] -- loaded before the ring wait of the iteration that finishes
// it, so its latency overlaps the stencil -- give
//     out = fma(dt, fma(c3, u*u*u, fma(c1, u, L)), u)      (FP32, then rounded to storage).
#pragma once

#include "stream.cuh"
#include "var.cuh"

namespace gst {

struct ReactionEpi {
    struct Params {
        float dt, c1, c3;
    };
    template <int VY, int VX> struct Regs {
        float u[VY][VX];  // u^t at the output cells
    };
    template <typename T, int VY, int VX>
    __device__ __forceinline__ static void prefetch(const StreamParams<T> &p, const Params &,
                                                    int zo, int oy, int ox, bool vec,
                                                    int vy_valid, Regs<VY, VX> &r) {
        const int nvalid = p.nx - ox;
#pragma unroll
        for (int vy = 0; vy < VY; ++vy) {
            if (vy >= vy_valid) break;
            const size_t base = ((size_t)zo * p.ny + oy + vy) * p.nx + ox;
            load_cells<T, VX>(p.in + base, vec, nvalid, r.u[vy]);
        }
    }
    template <typename T, int VY, int VX>
    __device__ __forceinline__ static void apply(const StreamParams<T> &p, const Params &e,
                                                 int zo, int oy, int ox, bool vec, int vy_valid,
                                                 const Regs<VY, VX> &r,
                                                 const float (&L)[VY][VX]) {
        const int nvalid = p.nx - ox;
#pragma unroll
        for (int vy = 0; vy < VY; ++vy) {
            if (vy >= vy_valid) break;
            float o[VX];
#pragma unroll
            for (int i = 0; i < VX; ++i) {
                const float u = r.u[vy][i];
                const float rate = fmaf(e.c3, u * u * u, fmaf(e.c1, u, L[vy][i]));
                o[i] = fmaf(e.dt, rate, u);
            }
            store_cells<T, VX>(p.out + ((size_t)zo * p.ny + oy + vy) * p.nx + ox, vec, nvalid, o);
        }
    }
};

}  // namespace gst
