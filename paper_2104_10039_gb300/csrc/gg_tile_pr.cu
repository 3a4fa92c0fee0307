// gg_tile_pr.cu - PageRank instantiations of the tile engine: the pull
// gather of approximate / accurate iterations and the correction iteration.
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

cudaError_t launch_tile_pr(int kind, const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    if (kind == K_GATHER) {
        int g = occupancy_grid<GG_APP_PAGERANK, K_GATHER>(num_sms);
        g = g < max_tiles ? g : (max_tiles > 0 ? max_tiles : 1);
        k_tile<GG_APP_PAGERANK, K_GATHER><<<g, kThreads, 0, s>>>(a);
    } else {
        int g = occupancy_grid<GG_APP_PAGERANK, K_CORRECT>(num_sms);
        g = g < max_tiles ? g : (max_tiles > 0 ? max_tiles : 1);
        k_tile<GG_APP_PAGERANK, K_CORRECT><<<g, kThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace gg
