// Prints the operations of the host-buffer wavefront (paper_2609_06694_gb300/csrc/wavefront.h)
// one per line -- "kind slab t a b" -- for the arguments nz R periodic steps nslab zb[0..nslab].
// Built and run by tests/test_wavefront_cpu.py, which replays the schedule plane by plane.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_2609_06694_gb300/csrc/wavefront.h"

int main(int argc, char **argv) {
    if (argc < 6) return 2;
    const long long nz = std::atoll(argv[1]), R = std::atoll(argv[2]);
    const bool periodic = std::atoi(argv[3]) != 0;
    const int steps = std::atoi(argv[4]), nslab = std::atoi(argv[5]);
    if (argc != 6 + nslab + 1) return 2;
    std::vector<int64_t> zb(nslab + 1);
    for (int k = 0; k <= nslab; ++k) zb[k] = std::atoll(argv[6 + k]);
    return gst::wavefront_schedule(nz, R, periodic, steps, zb.data(), nslab,
                                   [](int kind, int slab, int t, int64_t a, int64_t b) {
                                       std::printf("%d %d %d %lld %lld\n", kind, slab, t,
                                                   (long long)a, (long long)b);
                                       return 0;
                                   });
}
