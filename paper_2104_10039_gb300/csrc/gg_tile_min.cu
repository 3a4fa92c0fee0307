// gg_tile_min.cu - SSSP, BFS and CC instantiations of the tile engine (pull
// gather and correction on a min accumulator) and the edge sampler.
#include "gg_tile.cuh"

namespace gg {

template <int APP, int KIND>
static int occupancy_grid(int num_sms)
{
    static int blocks = 0;
    if (blocks == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_tile<APP, KIND>, kThreads, 0) != cudaSuccess || b < 1)
            b = 1;
        blocks = b;
    }
    return blocks * num_sms;
}

template <int APP, int KIND>
static void launch_one(const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    int g = occupancy_grid<APP, KIND>(num_sms);
    g = g < max_tiles ? g : (max_tiles > 0 ? max_tiles : 1);
    k_tile<APP, KIND><<<g, kThreads, 0, s>>>(a);
}

cudaError_t launch_tile_min(int app, int kind, const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    switch (app * 2 + (kind == K_CORRECT ? 1 : 0)) {
    case GG_APP_SSSP * 2: launch_one<GG_APP_SSSP, K_GATHER>(a, max_tiles, num_sms, s); break;
    case GG_APP_SSSP * 2 + 1: launch_one<GG_APP_SSSP, K_CORRECT>(a, max_tiles, num_sms, s); break;
    case GG_APP_BFS * 2: launch_one<GG_APP_BFS, K_GATHER>(a, max_tiles, num_sms, s); break;
    case GG_APP_BFS * 2 + 1: launch_one<GG_APP_BFS, K_CORRECT>(a, max_tiles, num_sms, s); break;
    case GG_APP_CC * 2: launch_one<GG_APP_CC, K_GATHER>(a, max_tiles, num_sms, s); break;
    case GG_APP_CC * 2 + 1: launch_one<GG_APP_CC, K_CORRECT>(a, max_tiles, num_sms, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Sampling (Sec. 3.4) reuses the tile walk over the full in-edge list: the
// hash decides each flag, and the active arcs are packed. The value type of
// the instantiation is irrelevant (no gather).
cudaError_t launch_tile_sample(const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    launch_one<GG_APP_CC, K_SAMPLE>(a, max_tiles, num_sms, s);
    return cudaGetLastError();
}

}  // namespace gg
