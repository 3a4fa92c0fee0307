// gg_tile_pr.cu - PageRank instantiations of the tile engine: the pull
// gather of approximate / accurate iterations and the correction iteration.
#include "gg_tile_launch.cuh"

namespace gg {

cudaError_t launch_tile_pr(int kind, const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    if (kind == K_GATHER) return launch_gather<GG_APP_PAGERANK>(a, max_tiles, num_sms, s);
    return launch_correction<GG_APP_PAGERANK>(a, max_tiles, num_sms, s);
}

cudaError_t launch_fixup_pr(const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    return launch_fixup_app<GG_APP_PAGERANK>(a, max_tiles, num_sms, s);
}

}  // namespace gg
