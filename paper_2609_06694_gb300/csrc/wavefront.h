// The schedule of stencil_apply_host's multi-sweep wavefront over z (host code only, no CUDA:
// plan.cpp issues the operations, and the CPU tests replay the same schedule plane by plane).
//
// The input arrives in slabs [zb[k], zb[k + 1]).  Sweep t of output planes [a, b) reads sweep
// t - 1 (the input for t = 1) on [a - R, b + R), so once the input planes [0, A) have landed,
// sweep 1 can run up to A - R, sweep 2 up to A - 2R, ...; each sweep t keeps a frontier F[t].
// A zero-Dirichlet grid fills [0, F[t]) and reaches nz with the last slab.  On a periodic grid
// the planes within tR of either end of sweep t read wrapped planes of sweep t - 1: its band is
// [tR, nz - tR), and [F[t], nz) and [0, tR) follow once every band is complete, sweep by sweep.
// The finished planes of the last sweep are copied out as soon as they are done.  Run in the
// order emitted, on buffers that alternate between sweeps (sweep t writes the buffer sweep
// t - 2 wrote), no sweep overwrites planes that the sweep before it still reads:
// F[t + 2] <= F[t + 1] - R.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace gst {

enum WaveOpKind : int {
    kWaveWaitInput = 0,  // wait until input slab `slab` has landed
    kWaveSweep = 1,      // sweep t on output planes [a, b)
    kWaveCopyOut = 2,    // copy planes [a, b) of the last sweep out
};

// Calls op(kind, slab, t, a, b) for every operation in issue order; stops at the first call
// that returns nonzero and returns that value (0 when the schedule is complete).
template <class Op>
int wavefront_schedule(int64_t nz, int64_t R, bool periodic, int steps, const int64_t *zb,
                       int nslab, Op &&op) {
    std::vector<int64_t> lo(steps + 1), hi(steps + 1), F(steps + 1);
    for (int t = 1; t <= steps; ++t) {
        lo[t] = periodic ? std::min<int64_t>(t * R, nz) : 0;
        hi[t] = periodic ? std::max<int64_t>(lo[t], nz - t * R) : nz;
        F[t] = lo[t];
    }
    int rc = 0;
    int64_t sent = lo[steps];  // the last sweep's planes [lo, sent) are on their way out
    for (int k = 0; k < nslab; ++k) {
        if ((rc = op(kWaveWaitInput, k, 0, zb[k], zb[k + 1]))) return rc;
        int64_t avail = zb[k + 1];  // frontier of the values the next sweep reads
        for (int t = 1; t <= steps; ++t) {
            const int64_t target = periodic ? std::min(hi[t], std::max(lo[t], avail - R))
                                            : (avail >= nz ? nz : std::max<int64_t>(0, avail - R));
            if (target > F[t]) {
                if ((rc = op(kWaveSweep, k, t, F[t], target))) return rc;
                F[t] = target;
            }
            avail = F[t];
        }
        if (F[steps] > sent) {
            if ((rc = op(kWaveCopyOut, k, steps, sent, F[steps]))) return rc;
            sent = F[steps];
        }
    }
    if (periodic) {
        for (int t = 1; t <= steps; ++t) {
            if (nz > F[t] && (rc = op(kWaveSweep, nslab, t, F[t], nz))) return rc;
            if (lo[t] > 0 && (rc = op(kWaveSweep, nslab, t, 0, lo[t]))) return rc;
        }
        if (nz > sent && (rc = op(kWaveCopyOut, nslab, steps, sent, nz))) return rc;
        if (lo[steps] > 0 && (rc = op(kWaveCopyOut, nslab, steps, 0, lo[steps]))) return rc;
    }
    return 0;
}

}  // namespace gst
