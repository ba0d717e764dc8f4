// Launchers of the reaction-diffusion kernel (reaction.cuh): the streaming kernel with the
// reaction epilogue, one output row per thread, for the star sets of radius 1, 2 and 4 and the
// radius-1 box, 2D and 3D.
#pragma once

#include "internal.h"
#include "reaction.cuh"
#include "stream_launch.cuh"

namespace gst {

template <typename T, int NDIM, int SHAPE>
int launch_reaction_r(const StreamLaunch &L, const ReactionEpi::Params &e) {
    if constexpr (SHAPE == kStar) {
        if (L.radius == 1) return launch_stream_t<T, NDIM, SHAPE, 1, 1, ReactionEpi>(L, e);
        if (L.radius == 2) return launch_stream_t<T, NDIM, SHAPE, 2, 1, ReactionEpi>(L, e);
        if (L.radius == 4) return launch_stream_t<T, NDIM, SHAPE, 4, 1, ReactionEpi>(L, e);
    } else {
        if (L.radius == 1) return launch_stream_t<T, NDIM, SHAPE, 1, 1, ReactionEpi>(L, e);
    }
    return -2;
}

template <typename T> int launch_reaction_t(const StreamLaunch &L, float dt, float c1, float c3) {
    const ReactionEpi::Params e{dt, c1, c3};
    if (L.vec_y != 1) return -1;
    if (L.ndim == 3) {
        if (L.shape == kStar) return launch_reaction_r<T, 3, kStar>(L, e);
        if (L.shape == kBox) return launch_reaction_r<T, 3, kBox>(L, e);
    } else if (L.ndim == 2) {
        if (L.shape == kStar) return launch_reaction_r<T, 2, kStar>(L, e);
        if (L.shape == kBox) return launch_reaction_r<T, 2, kBox>(L, e);
    }
    return -2;
}

}  // namespace gst
